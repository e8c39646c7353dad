// pct_grad.cu -- kernels for gradient-based reconstruction beside DROP:
//   * isotropic total variation TV(x) = sum_v sqrt(|D+ x|_v^2 + eps^2) and its
//     gradient (forward differences, zero difference at the last index of an
//     axis), gathered per voxel so that no atomics are needed;
//   * one Adam step (Kingma & Ba) over a parameter vector.
// The paper solves A x = b with DROP only; these kernels let a caller minimise
// ||A x - b||^2 + w TV(x) with the projector of pct_forward / pct_adjoint.
#include <cmath>

#include "pct_internal.h"

namespace pct {

namespace {

constexpr int kTvCta = 256;

struct TvGrid {
    int nx, ny, nz;
    __device__ __forceinline__ int at(int ix, int iy, int iz) const { return ix + nx * (iy + ny * iz); }
};

// Forward differences at voxel (ix, iy, iz) and the stencil norm there.
__device__ __forceinline__ float tv_norm(const float* __restrict__ x, const TvGrid& g, int ix, int iy,
                                         int iz, float eps2, float& dx, float& dy, float& dz)
{
    const int v = g.at(ix, iy, iz);
    const float xv = __ldg(x + v);
    dx = ix + 1 < g.nx ? __ldg(x + v + 1) - xv : 0.f;
    dy = iy + 1 < g.ny ? __ldg(x + v + g.nx) - xv : 0.f;
    dz = iz + 1 < g.nz ? __ldg(x + v + g.nx * g.ny) - xv : 0.f;
    return sqrtf(fmaf(dx, dx, fmaf(dy, dy, fmaf(dz, dz, eps2))));
}

__global__ void __launch_bounds__(kTvCta)
k_tv(const float* __restrict__ x, TvGrid g, float eps, float* __restrict__ grad, double* value)
{
    __shared__ double part[kTvCta / 32];
    const int64_t n = (int64_t)g.nx * g.ny * g.nz;
    const int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const float eps2 = eps * eps;
    double mine = 0.0;
    if (v < n) {
        const int ix = (int)(v % g.nx), iy = (int)((v / g.nx) % g.ny), iz = (int)(v / ((int64_t)g.nx * g.ny));
        float dx, dy, dz;
        const float nv = tv_norm(x, g, ix, iy, iz, eps2, dx, dy, dz);
        mine = nv;
        // d/dx_v of the norm at v, and of the norms at the three lower neighbours
        float gv = -(dx + dy + dz) / nv;
        float ax, ay, az;
        if (ix > 0) {
            const float nn = tv_norm(x, g, ix - 1, iy, iz, eps2, ax, ay, az);
            gv += ax / nn;
        }
        if (iy > 0) {
            const float nn = tv_norm(x, g, ix, iy - 1, iz, eps2, ax, ay, az);
            gv += ay / nn;
        }
        if (iz > 0) {
            const float nn = tv_norm(x, g, ix, iy, iz - 1, eps2, ax, ay, az);
            gv += az / nn;
        }
        grad[v] = gv;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mine += __shfl_xor_sync(0xffffffffu, mine, o);
    if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = mine;
    __syncthreads();
    if (threadIdx.x < 32) {
        double s = threadIdx.x < (blockDim.x >> 5) ? part[threadIdx.x] : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (threadIdx.x == 0) atomicAdd(value, s);
    }
}

__global__ void k_adam(float* __restrict__ x, const float* __restrict__ g, float* __restrict__ m,
                       float* __restrict__ v, int64_t n, float lr, float b1, float b2, float eps,
                       float c1, float c2)
{
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += stride) {
        const float gk = g[k];
        const float mk = fmaf(b1, m[k], (1.f - b1) * gk);
        const float vk = fmaf(b2, v[k], (1.f - b2) * gk * gk);
        m[k] = mk;
        v[k] = vk;
        x[k] -= lr * (mk * c1) / (sqrtf(vk * c2) + eps);
    }
}

}  // namespace

cudaError_t launch_tv(const Launch& L, const float* x, int nx, int ny, int nz, float eps, float* grad,
                      double* value)
{
    const int64_t n = (int64_t)nx * ny * nz;
    cudaError_t e = cudaMemsetAsync(value, 0, sizeof(double), L.stream);
    if (e != cudaSuccess) return e;
    k_tv<<<(unsigned)((n + kTvCta - 1) / kTvCta), kTvCta, 0, L.stream>>>(x, TvGrid{nx, ny, nz}, eps,
                                                                       grad, value);
    ++*L.launches;
    return cudaGetLastError();
}

cudaError_t launch_adam(const Launch& L, float* x, const float* g, float* m, float* v, int64_t n,
                        float lr, float b1, float b2, float eps, int step)
{
    if (n <= 0) return cudaSuccess;
    // bias corrections 1/(1 - b^t), evaluated on the host in double
    const float c1 = (float)(1.0 / (1.0 - std::pow((double)b1, step)));
    const float c2 = (float)(1.0 / (1.0 - std::pow((double)b2, step)));
    int64_t blocks = (n + 255) / 256;
    if (blocks > 148 * 16) blocks = 148 * 16;
    k_adam<<<(unsigned)blocks, 256, 0, L.stream>>>(x, g, m, v, n, lr, b1, b2, eps, c1, c2);
    ++*L.launches;
    return cudaGetLastError();
}

}  // namespace pct
