// pct_batch.cu -- many independent DROP reconstructions (scans) in one
// persistent cooperative launch.
//
// Each scan owns a contiguous range of CTAs, sized in proportion to its work
// (protons x iterations).  The CTAs of a scan run the scan's DROP blocks in
// order (Sec. IV-B): one warp per proton for the block step, a barrier among
// the scan's CTAs, the block apply, another barrier.  Scans never wait on each
// other.  The launch is cooperative, so all CTAs are resident together and the
// per-scan barriers cannot wait for a CTA that is not running.  Every barrier
// wait is bounded: after `spin_limit` polls the waiting CTA sets a flag, marks
// the scan aborted and returns, so a lost arrival ends the kernel with an error
// instead of hanging it.
//
// x and the accumulator are rewritten inside the launch by other CTAs, so they
// are read through L2 only (ld.global.cg) and written back the same way.
//
// Within a block step the scan's warps take one or two protons by index and
// then chunks from the scan's work counter, so that the barrier after the step
// does not wait for one unlucky warp; the scan's first thread resets the
// counter between the two barriers of the block.
#include "pct_batch.h"
#include "pct_warp.cuh"

namespace pct {

namespace {

constexpr int kBatchRunSlots = 24;
constexpr int kBatchGrab = 2;

__device__ __forceinline__ bool scan_barrier(const ScanDesc& d, int* abort_flag, unsigned* flags,
                                             int spin_limit, int extra_target)
{
    __shared__ int ok;   // one decision for the whole CTA
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        const unsigned old = atomicAdd(d.bar, 1u);
        const unsigned target = (old / (unsigned)d.ncta + 1u) * (unsigned)d.ncta + (unsigned)extra_target;
        int spins = 0;
        while (true) {
            const unsigned now = *(volatile unsigned*)d.bar;
            if (now >= target) break;
            if (*(volatile int*)abort_flag) break;
            if (++spins > spin_limit) {
                atomicOr(flags, kFlagBarrierTimeout);
                atomicExch(abort_flag, 1);
                break;
            }
            __nanosleep(64);
        }
        __threadfence();
        ok = *(volatile int*)abort_flag == 0;
    }
    __syncthreads();
    return ok != 0;
}

// G = lanes per proton: 32 (one proton per warp) or 16 (two per warp).
template <int G>
__global__ void __launch_bounds__(256, 3)
k_drop_batch(const ScanDesc* __restrict__ scans, int nscan, unsigned* flags, int spin_limit,
             int test_unreachable)
{
    constexpr int kPerWarp = kWarp / G;
    extern __shared__ unsigned char smem[];
    int s = 0;
    while (s + 1 < nscan && (int)blockIdx.x >= scans[s + 1].cta0) ++s;
    const ScanDesc d = scans[s];
    if ((int)blockIdx.x >= d.cta0 + d.ncta) return;   // spare CTA beyond the last scan
    int* abort_flag = d.abort;
    const int warps = blockDim.x >> 5;
    const int warp_in_scan = ((int)blockIdx.x - d.cta0) * warps + (threadIdx.x >> 5);
    const int nwarp = d.ncta * warps;
    const int tid_in_scan = ((int)blockIdx.x - d.cta0) * blockDim.x + threadIdx.x;
    const int nthr = d.ncta * blockDim.x;
    const RunSlots slots{(int2*)(smem + (size_t)(threadIdx.x >> 5) * kBatchRunSlots * kWarp * 8)};
    const RecView rv{d.rec, d.stride};
    // only the first barrier of scan 0 is made unreachable by the test option
    int extra = (test_unreachable && s == 0) ? 1 : 0;
    const int lane = threadIdx.x & 31;
    const int sub = lane / G;   // which proton of the warp's unit this lane's group takes
    for (int it = 0; it < d.iters; ++it) {
        for (int64_t first = 0; first < d.n; first += d.block) {
            const int64_t count = d.block < d.n - first ? d.block : d.n - first;
            const int64_t units = (count + kPerWarp - 1) / kPerWarp;   // kPerWarp protons each
            const int per = units >= (int64_t)kBatchGrab * nwarp ? kBatchGrab : 1;
            const int64_t stat = (int64_t)nwarp * per;   // units assigned by index
            int64_t base = (int64_t)warp_in_scan * per, end = base + per;
            while (base < units) {
                end = end < units ? end : units;
                for (int64_t u = base; u < end; ++u) {
                    const int64_t p = u * kPerWarp + sub;
                    const int64_t i = first + p;
                    Path P;
                    if (kPerWarp == 1) {
                        if (!load_path(rv, i, d.mc, P)) continue;
                    } else {
                        // both groups of the warp take part in the walk's shuffles; a
                        // group without a valid proton walks nothing
                        __syncwarp();
                        if (!(p < count && load_path(rv, i, d.mc, P))) {
                            P = Path{};
                            P.nseg = 0;
                        }
                    }
                    LaneWalk w;
                    float sv, q;
                    warp_walk<kBatchRunSlots, true, true, G>(P, d.mc, d.g, d.mask, d.x, flags, slots,
                                                             d.mc.cmin, w, sv, q);
                    if (!(q > 0.f)) continue;
                    const float r = (rv.get(R_B, i) - sv) / q;
                    float2* acc = d.acc;
                    replay_runs<kBatchRunSlots>(P, d.mc, d.g, d.mask, flags, slots, w, [&](int j, float l) {
                        atomicAdd(acc + j, make_float2(l * r, 1.f));
                    });
                }
                if (stat >= units) break;
                unsigned long long got = 0;
                if (lane == 0) got = atomicAdd(d.next, (unsigned long long)kBatchGrab);
                base = stat + (int64_t)__shfl_sync(0xffffffffu, got, 0);
                end = base + kBatchGrab;
            }
            if (!scan_barrier(d, abort_flag, flags, spin_limit, extra)) return;
            extra = 0;
            // every warp of the scan is past its block step: reset the counter for
            // the next one (ordered before it by the barrier below)
            if (tid_in_scan == 0) atomicExch(d.next, 0ull);
            for (int64_t j = tid_in_scan; j < d.n_vox; j += nthr) {
                const float2 a = __ldcg(d.acc + j);
                if (a.y > 0.f) {
                    __stcg(d.x + j, fmaf(d.lambda, a.x / a.y, __ldcg(d.x + j)));
                    __stcg(d.acc + j, make_float2(0.f, 0.f));
                }
            }
            if (!scan_barrier(d, abort_flag, flags, spin_limit, 0)) return;
        }
    }
}

}  // namespace

size_t batch_smem(int cta)
{
    return (size_t)(cta / kWarp) * kBatchRunSlots * kWarp * 8;
}

namespace {

const void* batch_kernel(int lanes)
{
    return lanes == 16 ? (const void*)k_drop_batch<16> : (const void*)k_drop_batch<32>;
}

}  // namespace

cudaError_t batch_max_ctas(int cta, int lanes, int device, int* out)
{
    int per_sm = 0, sms = 0;
    const void* k = batch_kernel(lanes);
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)batch_smem(256));
    if (e != cudaSuccess) return e;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, cta, batch_smem(cta));
    if (e != cudaSuccess) return e;
    e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
    if (e != cudaSuccess) return e;
    *out = per_sm * sms;
    return cudaSuccess;
}

cudaError_t launch_drop_batch(const Launch& L, const ScanDesc* scans_dev, int nscan, int total_ctas,
                              int cta, int lanes, unsigned* flags, int spin_limit, int test_unreachable)
{
    void* args[] = {(void*)&scans_dev, (void*)&nscan, (void*)&flags, (void*)&spin_limit,
                    (void*)&test_unreachable};
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)total_ctas);
    cfg.blockDim = dim3((unsigned)cta);
    cfg.dynamicSmemBytes = batch_smem(cta);
    cfg.stream = L.stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    cudaError_t e = cudaLaunchKernelExC(&cfg, batch_kernel(lanes), args);
    ++*L.launches;
    return e;
}

}  // namespace pct
