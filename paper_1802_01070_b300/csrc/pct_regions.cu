// pct_regions.cu -- the image regions of the paper's Algorithm 1
// (arXiv:1802.01070, Sec. III) on one GPU: which protons belong to a region.
//
// The paper splits the volume along z into overlapping regions and associates
// each proton with the image region "entered to and exited from".  Here a
// proton with a hull path belongs to a region when the slices of both its hull
// entry point and its hull exit point lie in the region's extended slice range
// (a point on the grid's lowest or highest face counts in the first or last
// slice); both points come from the proton's record (the straight tracker
// lines followed to the full volume's hull), so every region walks the same
// MLP paths as the full-volume solve, restricted to its slab.
#include "pct_internal.h"

namespace pct {

namespace {

constexpr int kRegionCta = 256;

__device__ __forceinline__ int slice_of(double z, double oz, double dz, int nz)
{
    const double s = floor((z - oz) / dz);
    return s < 0.0 ? 0 : (s > (double)(nz - 1) ? nz - 1 : (int)s);
}

__global__ void __launch_bounds__(kRegionCta)
k_region_flags(const float* __restrict__ rec, int64_t stride, int64_t n, double oz, double dz, int nz, int lo,
               int hi, uint8_t* __restrict__ flag)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    bool in = false;
    if (rec[R_L * stride + i] > 0.f) {
        const int s0 = slice_of((double)rec[R_V0 * stride + i], oz, dz, nz);
        const int s2 = slice_of((double)rec[R_V2 * stride + i], oz, dz, nz);
        in = s0 >= lo && s0 < hi && s2 >= lo && s2 < hi;
    }
    flag[i] = in ? 1 : 0;
}

}  // namespace

cudaError_t launch_region_flags(const Launch& L, const float* rec, int64_t stride, int64_t n, const GridC& g,
                                int lo, int hi, uint8_t* flag)
{
    if (n <= 0) return cudaSuccess;
    k_region_flags<<<(unsigned)((n + kRegionCta - 1) / kRegionCta), kRegionCta, 0, L.stream>>>(
        rec, stride, n, (double)g.oz, (double)g.dz, g.nz, lo, hi, flag);
    ++*L.launches;
    return cudaGetLastError();
}

}  // namespace pct
