// pct_fbp.cu -- filtered back-projection (FBP) of the loaded proton
// histories: the initial iterate of the solve (arXiv:1802.01070, Sec. I: the
// FBP image is the initial iterate).  The paper gives no detail; the reading
// implemented is the textbook parallel-beam FBP applied slice by slice to
// binned list-mode data:
//
//   sinogram:  p[a, l, k] = mean WEPL of the protons in bin (angle a, v bin l,
//              t bin k) of pct_bins.cuh, 0 for an empty bin;
//   filter:    q[k] = dt sum_m p[m] h[k - m] along t, h the band-limited ramp
//              kernel h[0] = 1/(4 dt^2), h[odd n] = -1/(pi^2 n^2 dt^2), 0 else;
//   back-projection: voxel centre (x, y, z) in slice l = floor((z - v_min)/dv):
//              (pi / n_angle) sum_a q_a(-x sin phi_a + y cos phi_a), q_a linear
//              between bin centres, 0 beyond; phi_a = a angle_step.
//
// Kernels: one thread per proton for the bin sums (FP64 atomics), one CTA per
// sinogram row for the filter (the row in shared memory, FP64 sums), one
// thread per voxel for the back-projection (FP32, the angle table in shared
// memory, the filtered sinogram read through L1/L2: 4 B per bin, a few MB).
#include "pct_internal.h"

namespace pct {

namespace {

constexpr int kFbpCta = 256;
constexpr int kFilterCta = 256;
constexpr int kMaxAngles = 4096;   // angle table in shared memory (32 KB)

__global__ void __launch_bounds__(kFbpCta)
k_fbp_sum(ProtonBins P, const float* __restrict__ h, int64_t stride, int64_t n, unsigned* __restrict__ cnt,
          double* __restrict__ sum)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int b = proton_bin(P, h[H_INX * stride + i], h[H_INY * stride + i], h[H_INZ * stride + i],
                             h[H_OUTX * stride + i], h[H_OUTY * stride + i], h[H_OUTZ * stride + i],
                             h[H_PHI * stride + i]);
    if (b < 0) return;
    atomicAdd(cnt + b, 1u);
    atomicAdd(sum + b, (double)h[H_WEPL * stride + i]);
}

// One CTA per sinogram row (angle, v bin): mean WEPL of the row's bins in
// shared memory, then each thread filters some of the row's bins.
__global__ void __launch_bounds__(kFilterCta)
k_fbp_filter(int n_t, double dt, const unsigned* __restrict__ cnt, const double* __restrict__ sum,
             float* __restrict__ q)
{
    extern __shared__ double row[];
    const int64_t base = (int64_t)blockIdx.x * n_t;
    for (int k = threadIdx.x; k < n_t; k += blockDim.x) {
        const unsigned c = cnt[base + k];
        row[k] = c ? sum[base + k] / (double)c : 0.0;
    }
    __syncthreads();
    const double h0 = 1.0 / (4.0 * dt * dt);
    const double ho = -1.0 / (M_PI * M_PI * dt * dt);
    for (int k = threadIdx.x; k < n_t; k += blockDim.x) {
        double acc = h0 * row[k];
        // odd offsets n = k - m only
        for (int m = k - 1; m >= 0; m -= 2) {
            const double nn = (double)(k - m);
            acc += ho / (nn * nn) * row[m];
        }
        for (int m = k + 1; m < n_t; m += 2) {
            const double nn = (double)(m - k);
            acc += ho / (nn * nn) * row[m];
        }
        q[base + k] = (float)(dt * acc);
    }
}

__global__ void __launch_bounds__(kFbpCta)
k_fbp_backproject(ProtonBins P, GridC g, const uint8_t* __restrict__ hull, const float* __restrict__ q,
                  float* __restrict__ x)
{
    __shared__ float2 sc[kMaxAngles];
    for (int a = threadIdx.x; a < P.n_angle; a += blockDim.x) {
        double s, c;
        sincos((double)a * P.angle_step, &s, &c);
        sc[a] = make_float2((float)s, (float)c);
    }
    __syncthreads();
    const int64_t n_vox = (int64_t)g.nx * g.ny * g.nz;
    const int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (j >= n_vox) return;
    if (!hull[j]) {
        x[j] = 0.f;
        return;
    }
    const int ix = (int)(j % g.nx);
    const int iy = (int)((j / g.nx) % g.ny);
    const int iz = (int)(j / ((int64_t)g.nx * g.ny));
    const double zc = (double)g.oz + ((double)iz + 0.5) * (double)g.dz;
    const double lf = floor((zc - P.v_min) / P.dv);
    if (!(lf >= 0.0 && lf < (double)P.n_v)) {
        x[j] = 0.f;
        return;
    }
    const int l = (int)lf;
    const float xc = (float)((double)g.ox + ((double)ix + 0.5) * (double)g.dx);
    const float yc = (float)((double)g.oy + ((double)iy + 0.5) * (double)g.dy);
    const float inv_dt = (float)(1.0 / P.dt);
    const float off = (float)(-P.t_min / P.dt - 0.5);
    float acc = 0.f;
    for (int a = 0; a < P.n_angle; ++a) {
        const float2 s_c = sc[a];
        const float t = fmaf(yc, s_c.y, -xc * s_c.x);
        const float f = fmaf(t, inv_dt, off);
        const float k0f = floorf(f);
        const float w = f - k0f;
        const int k0 = (int)k0f;
        const float* r = q + ((int64_t)a * P.n_v + l) * P.n_t;
        const float v0 = (k0 >= 0 && k0 < P.n_t) ? __ldg(r + k0) : 0.f;
        const float v1 = (k0 + 1 >= 0 && k0 + 1 < P.n_t) ? __ldg(r + k0 + 1) : 0.f;
        acc += fmaf(w, v1 - v0, v0);
    }
    x[j] = acc * (float)(M_PI / (double)P.n_angle);
}

}  // namespace

int fbp_max_angles()
{
    return kMaxAngles;
}

cudaError_t launch_fbp(const Launch& L, const ProtonBins& P, const GridC& g, const uint8_t* hull,
                       const float* hist, int64_t stride, int64_t n, unsigned* cnt, double* sum, float* q,
                       float* x)
{
    const int64_t nb = (int64_t)P.n_angle * P.n_t * P.n_v;
    cudaError_t e = cudaMemsetAsync(cnt, 0, (size_t)nb * sizeof(unsigned), L.stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(sum, 0, (size_t)nb * sizeof(double), L.stream);
    if (e != cudaSuccess) return e;
    if (n > 0) {
        k_fbp_sum<<<(unsigned)((n + kFbpCta - 1) / kFbpCta), kFbpCta, 0, L.stream>>>(P, hist, stride, n, cnt, sum);
        ++*L.launches;
    }
    const size_t smem = (size_t)P.n_t * sizeof(double);
    if (smem > 48 * 1024) {
        e = cudaFuncSetAttribute(k_fbp_filter, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    k_fbp_filter<<<(unsigned)((int64_t)P.n_angle * P.n_v), kFilterCta, smem, L.stream>>>(P.n_t, P.dt, cnt,
                                                                                          sum, q);
    const int64_t n_vox = (int64_t)g.nx * g.ny * g.nz;
    k_fbp_backproject<<<(unsigned)((n_vox + kFbpCta - 1) / kFbpCta), kFbpCta, 0, L.stream>>>(P, g, hull, q, x);
    *L.launches += 2;
    return cudaGetLastError();
}

}  // namespace pct
