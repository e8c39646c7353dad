// pct_noalloc.cu -- pct_solve_noalloc: the DROP reconstruction of pct_solve for
// callers that cannot allocate device memory.  Every scratch buffer it needs
// lives in the fixed-size device arrays below, which the CUDA runtime places in
// the library's module image when the library is loaded on a device; the call
// itself never allocates or frees device memory.
#include <cmath>
#include <cstring>
#include <mutex>
#include <string>

#include "pct.h"
#include "pct_internal.h"

using namespace pct;

namespace {

constexpr int kMaxDevices = 64;

// Scratch, shared by every call on a device (contents persist between calls).
static __device__ __align__(256) float g_hist[H_NF * PCT_NOALLOC_MAX_PROTONS];
static __device__ __align__(256) float g_rec[R_NF * PCT_NOALLOC_MAX_PROTONS];
static __device__ __align__(256) float2 g_acc[PCT_NOALLOC_MAX_VOXELS];
static __device__ __align__(256) float4 g_sig1[PCT_NOALLOC_MAX_SAMPLES + 1];
static __device__ __align__(256) unsigned g_flags[1];
static __device__ __align__(256) unsigned long long g_next[1];
static __device__ __align__(256) int64_t g_vidx[PCT_NOALLOC_MAX_PROTONS];
static __device__ __align__(256) int64_t g_boff[PCT_NOALLOC_MAX_PROTONS + 1];
static __device__ __align__(256) int64_t g_chunk[PCT_NOALLOC_MAX_PROTONS / kCompactChunk + 1];
static __device__ __align__(256) uint8_t g_dist[PCT_NOALLOC_MAX_VOXELS];
static __device__ __align__(256) uint8_t g_dist_tmp[PCT_NOALLOC_MAX_VOXELS];

struct Scratch {
    bool ready = false;
    float* hist = nullptr;
    float* rec = nullptr;
    float2* acc = nullptr;
    float4* sig1 = nullptr;
    unsigned* flags = nullptr;
    uint8_t* dist = nullptr;
    uint8_t* dist_tmp = nullptr;
    int64_t* vidx = nullptr;
    int64_t* boff = nullptr;
    int64_t* chunk = nullptr;
    unsigned long long* next = nullptr;
};

Scratch g_scratch[kMaxDevices];
std::mutex g_scratch_mu;

// This entry point has no context to hold a message: failures are reported by
// status alone (the message argument documents the cause in the source).
pct_status fail(pct_status s, const std::string&)
{
    return s;
}

// Every CUDA failure, a launch that lacks resources included, is PCT_ERR_CUDA:
// this call allocates nothing, so it never reports PCT_ERR_OOM.
pct_status cuda_fail(cudaError_t e, const char*)
{
    (void)e;
    cudaGetLastError();
    return PCT_ERR_CUDA;
}

// Device addresses of the scratch arrays for `device`, looked up once with the
// device current.  (In host code the array names are host-side stand-ins, not
// device addresses.)
pct_status scratch_for(int device, Scratch& out)
{
    if (device < 0 || device >= kMaxDevices) return fail(PCT_ERR_ARG, "device index out of range");
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    Scratch& s = g_scratch[device];
    if (!s.ready) {
        cudaError_t e;
        if ((e = cudaGetSymbolAddress((void**)&s.hist, g_hist)) != cudaSuccess ||
            (e = cudaGetSymbolAddress((void**)&s.rec, g_rec)) != cudaSuccess ||
            (e = cudaGetSymbolAddress((void**)&s.acc, g_acc)) != cudaSuccess ||
            (e = cudaGetSymbolAddress((void**)&s.sig1, g_sig1)) != cudaSuccess ||
            (e = cudaGetSymbolAddress((void**)&s.flags, g_flags)) != cudaSuccess ||
            (e = cudaGetSymbolAddress((void**)&s.dist, g_dist)) != cudaSuccess ||
            (e = cudaGetSymbolAddress((void**)&s.dist_tmp, g_dist_tmp)) != cudaSuccess ||
            (e = cudaGetSymbolAddress((void**)&s.vidx, g_vidx)) != cudaSuccess ||
            (e = cudaGetSymbolAddress((void**)&s.boff, g_boff)) != cudaSuccess ||
            (e = cudaGetSymbolAddress((void**)&s.chunk, g_chunk)) != cudaSuccess ||
            (e = cudaGetSymbolAddress((void**)&s.next, g_next)) != cudaSuccess)
            return cuda_fail(e, "scratch address lookup");
        s.ready = true;
    }
    out = s;
    return PCT_OK;
}

struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev)
    {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        if (prev != dev) cudaSetDevice(dev);
    }
    ~DeviceGuard()
    {
        if (prev >= 0) cudaSetDevice(prev);
    }
};

}  // namespace

extern "C" pct_status pct_solve_noalloc(const pct_grid* grid, const uint8_t* hull_mask, int64_t n,
                                        const float* const in_xyz[3], const float* const out_xyz[3],
                                        const float* const ang_in[2], const float* const ang_out[2],
                                        const float* gantry_rad, const float* wepl_mm, int32_t iters,
                                        float lambda, int64_t block_size, float* x, int device,
                                        void* cuda_stream)
{
    if (!grid || !hull_mask || !x) return fail(PCT_ERR_ARG, "null grid, hull mask or x");
    const pct_grid& G = *grid;
    if (G.nx < 1 || G.ny < 1 || G.nz < 1 || !(G.dx > 0.f) || !(G.dy > 0.f) || !(G.dz > 0.f) ||
        !std::isfinite(G.dx) || !std::isfinite(G.dy) || !std::isfinite(G.dz) ||
        !std::isfinite(G.ox) || !std::isfinite(G.oy) || !std::isfinite(G.oz))
        return fail(PCT_ERR_ARG, "invalid grid");
    const int64_t n_vox = (int64_t)G.nx * G.ny * G.nz;
    if (n_vox > PCT_NOALLOC_MAX_VOXELS)
        return fail(PCT_ERR_ARG, "grid has " + std::to_string(n_vox) + " voxels, the limit is " +
                                     std::to_string(PCT_NOALLOC_MAX_VOXELS));
    if (n < 0 || n > PCT_NOALLOC_MAX_PROTONS)
        return fail(PCT_ERR_ARG, "proton count " + std::to_string(n) + " outside 0.." +
                                     std::to_string(PCT_NOALLOC_MAX_PROTONS));
    if (iters < 0 || block_size < 1 || !std::isfinite(lambda))
        return fail(PCT_ERR_ARG, "iters < 0, block size < 1 or non-finite lambda");
    const float* src[H_NF] = {nullptr};
    if (n > 0) {
        if (!in_xyz || !out_xyz || !ang_in || !ang_out || !gantry_rad || !wepl_mm)
            return fail(PCT_ERR_ARG, "null history pointer");
        const float* s[H_NF] = {in_xyz[0], in_xyz[1], in_xyz[2], out_xyz[0], out_xyz[1], out_xyz[2],
                                ang_in[0], ang_in[1], ang_out[0], ang_out[1], gantry_rad, wepl_mm};
        for (int f = 0; f < H_NF; ++f) {
            if (!s[f]) return fail(PCT_ERR_ARG, "null history pointer");
            src[f] = s[f];
        }
    }
    // MLP sample table (same spacing rule as the context path: du = smallest voxel edge)
    const double du = std::fmin((double)G.dx, std::fmin((double)G.dy, (double)G.dz));
    const double diag = std::sqrt(std::pow((double)G.nx * G.dx, 2) + std::pow((double)G.ny * G.dy, 2) +
                                  std::pow((double)G.nz * G.dz, 2));
    const int kmax = (int)std::ceil(diag / du) + 3;
    if (kmax > PCT_NOALLOC_MAX_SAMPLES)
        return fail(PCT_ERR_ARG, "grid diagonal spans more than " +
                                     std::to_string(PCT_NOALLOC_MAX_SAMPLES) + " MLP samples");
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
        cudaGetLastError();
        return fail(PCT_ERR_ARG, "no such CUDA device");
    }
    DeviceGuard dg(device);
    Scratch S;
    pct_status st = scratch_for(device, S);
    if (st != PCT_OK) return st;
    cudaStream_t stream = (cudaStream_t)cuda_stream;
    static thread_local float4 tab[PCT_NOALLOC_MAX_SAMPLES + 1];
    mlp_sigma_table(du, kmax, tab);
    cudaError_t e = cudaMemcpyAsync(S.sig1, tab, sizeof(float4) * (size_t)(kmax + 1),
                                    cudaMemcpyHostToDevice, stream);
    if (e != cudaSuccess) return cuda_fail(e, "MLP table upload");
    if ((e = cudaMemsetAsync(S.flags, 0, sizeof(unsigned), stream)) != cudaSuccess)
        return cuda_fail(e, "flag clear");

    Geo geo;
    geo.g.nx = G.nx;
    geo.g.ny = G.ny;
    geo.g.nz = G.nz;
    geo.g.dx = G.dx;
    geo.g.dy = G.dy;
    geo.g.dz = G.dz;
    geo.g.ox = G.ox;
    geo.g.oy = G.oy;
    geo.g.oz = G.oz;
    geo.g.idx = 1.f / G.dx;
    geo.g.idy = 1.f / G.dy;
    geo.g.idz = 1.f / G.dz;
    geo.mc.du_mm = (float)du;
    geo.mc.du_cm = (float)(0.1 * du);
    geo.mc.dend_mm = (float)(1e-3 * du);
    for (int k = 0; k < 6; ++k) geo.mc.coef[k] = (float)kCoef200[k];
    geo.mc.sig1 = S.sig1;
    geo.mc.kmax = kmax;
    const double vdiag = std::sqrt((double)G.dx * G.dx + (double)G.dy * G.dy + (double)G.dz * G.dz);
    geo.mc.cmin = (int)std::floor(vdiag / du) + 1;
    geo.mask = hull_mask;
    geo.dist = S.dist;
    geo.flags = S.flags;
    int64_t launches = 0;
    const Launch L{stream, 256, &launches};
    const int64_t stride = PCT_NOALLOC_MAX_PROTONS;

    if (n > 0 && iters > 0) {
        for (int f = 0; f < H_NF; ++f) {
            e = cudaMemcpyAsync(S.hist + (size_t)f * stride, src[f], (size_t)n * sizeof(float),
                                cudaMemcpyDeviceToDevice, stream);
            if (e != cudaSuccess) return cuda_fail(e, "history copy");
        }
        if ((e = launch_hull_dist(L, hull_mask, G.nx, G.ny, G.nz, S.dist_tmp, S.dist)) != cudaSuccess)
            return cuda_fail(e, "hull distance map");
        if ((e = launch_prepare(L, geo, S.hist, stride, n, S.rec)) != cudaSuccess)
            return cuda_fail(e, "prepare kernel");
        if ((e = launch_compact(L, S.rec, stride, n, block_size, S.chunk, S.vidx, S.boff)) != cudaSuccess)
            return cuda_fail(e, "valid-proton lists");
        // the accumulator and the work counter must start at zero; every block
        // apply leaves them at zero
        if ((e = cudaMemsetAsync(S.acc, 0, (size_t)n_vox * sizeof(float2), stream)) != cudaSuccess ||
            (e = cudaMemsetAsync(S.next, 0, sizeof(unsigned long long), stream)) != cudaSuccess)
            return cuda_fail(e, "accumulator clear");
        for (int32_t it = 0; it < iters; ++it) {
            for (int64_t first = 0; first < n; first += block_size) {
                const int64_t count = block_size < n - first ? block_size : n - first;
                if ((e = launch_drop_fused(L, geo, S.rec, stride, S.vidx, S.boff, first / block_size, count, x,
                                           S.acc, S.next)) != cudaSuccess)
                    return cuda_fail(e, "DROP kernel");
                if ((e = launch_drop_apply(L, n_vox, hull_mask, x, S.acc, lambda, S.next)) != cudaSuccess)
                    return cuda_fail(e, "DROP apply kernel");
            }
        }
    }
    if ((e = cudaStreamSynchronize(stream)) != cudaSuccess) return cuda_fail(e, "stream");
    unsigned flags = 0;
    if ((e = cudaMemcpy(&flags, S.flags, sizeof flags, cudaMemcpyDeviceToHost)) != cudaSuccess)
        return cuda_fail(e, "flag read");
    if (flags) return fail(PCT_ERR_DEVICE, "device check failed (flags " + std::to_string(flags) + ")");
    return PCT_OK;
}
