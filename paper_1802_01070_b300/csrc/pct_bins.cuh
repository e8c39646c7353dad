// pct_bins.cuh -- the (gantry angle, t, v) bin of a proton, shared by the
// data-cleaning (pct_clean.cu) and FBP (pct_fbp.cu) kernels.  FP64 from the
// float32 tracker data: the angle bin is the nearest multiple of angle_step
// (mod n_angle); t and v are where the straight chord between the entry and
// exit tracker points crosses depth u = 0 of the proton's beam frame
// (arXiv:1802.01070 bins nothing itself; this is the usual list-mode binning).
// The library is compiled without implicit multiply-add contraction, so the
// products and sums round as written.
#pragma once

#include <cuda_runtime.h>
#include <math.h>

namespace pct {

struct ProtonBins {
    int n_angle, n_t, n_v;
    double angle_step, t_min, dt, v_min, dv;
};

// Linear bin (a * n_v + k_v) * n_t + k_t, or -1 outside the t or v bins.
__device__ __forceinline__ int proton_bin(const ProtonBins& P, double x0, double y0, double z0, double x1,
                                          double y1, double z1, double phi)
{
    double s, c;
    sincos(phi, &s, &c);
    const double u0 = x0 * c + y0 * s, t0 = -x0 * s + y0 * c;
    const double u1 = x1 * c + y1 * s, t1 = -x1 * s + y1 * c;
    const double w = -u0 / (u1 - u0);
    const double t = t0 + w * (t1 - t0);
    const double v = z0 + w * (z1 - z0);
    const double ka = floor(phi / P.angle_step + 0.5);
    const double kt = floor((t - P.t_min) / P.dt);
    const double kv = floor((v - P.v_min) / P.dv);
    if (!(kt >= 0.0 && kt < (double)P.n_t && kv >= 0.0 && kv < (double)P.n_v) || !isfinite(ka)) return -1;
    long long a = (long long)ka % P.n_angle;
    if (a < 0) a += P.n_angle;
    return (int)((a * P.n_v + (long long)kv) * P.n_t + (long long)kt);
}

}  // namespace pct
