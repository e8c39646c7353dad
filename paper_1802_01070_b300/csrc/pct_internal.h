// pct_internal.h -- private interface between the C ABI (pct_api.cu) and the
// kernel launchers (pct_kernels.cu).  Not installed, not part of the ABI.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "pct_device.cuh"

namespace pct {

// Device pointers of one loaded history set (12 SoA columns, stride floats apart):
// in_x, in_y, in_z, out_x, out_y, out_z, theta_in, psi_in, theta_out, psi_out, phi, wepl.
enum HistField { H_INX = 0, H_INY, H_INZ, H_OUTX, H_OUTY, H_OUTZ, H_THI, H_PSI, H_THO, H_PSO, H_PHI,
                 H_WEPL, H_NF };

struct Launch {
    cudaStream_t stream;
    int cta;              // threads per block for per-proton kernels
    int64_t* launches;    // launch counter to bump
};

struct Geo {
    GridC g;
    MlpC mc;
    const uint8_t* mask;  // device, nx*ny*nz bytes
    unsigned* flags;      // device error word
};

cudaError_t launch_prepare(const Launch& L, const Geo& G, const float* hist, int64_t stride,
                           int64_t n, float* rec);
cudaError_t launch_hull_states(const Launch& L, const float* rec, int64_t stride, int64_t first,
                               int64_t count, float* out);
cudaError_t launch_mlp_points(const Launch& L, const Geo& G, const float* rec, int64_t stride,
                              int64_t first, int64_t count, int32_t max_pts, float* out_xyz,
                              int32_t* out_npts);
cudaError_t launch_rows(const Launch& L, const Geo& G, const float* rec, int64_t stride,
                        int64_t first, int64_t count, int32_t max_nnz, int32_t* out_idx,
                        float* out_len, int32_t* out_nnz);
cudaError_t launch_forward(const Launch& L, const Geo& G, const float* rec, int64_t stride,
                           int64_t n, const float* x, float* y);
cudaError_t launch_adjoint(const Launch& L, const Geo& G, const float* rec, int64_t stride,
                           int64_t n, const float* y, float* g_out);
cudaError_t launch_drop_fused(const Launch& L, const Geo& G, const float* rec, int64_t stride,
                              int64_t first, int64_t count, const float* x, float2* acc);
cudaError_t launch_drop_apply(const Launch& L, int64_t n_vox, float* x, float2* acc, float lambda);

}  // namespace pct
