// pct_clean.cu -- data cleaning of the loaded proton histories: statistical
// outlier removal per (gantry angle, t, v) bin (arXiv:1802.01070, Sec. IV-A:
// the scans are reduced by identifying and removing statistical outliers
// before the solve).  The paper gives no detail; the reading implemented:
//
//   bin:   angle bin = nearest multiple of angle_step (mod n_angle); t, v = the
//          lateral and vertical position where the straight chord between the
//          entry and exit tracker points crosses depth u = 0 of the proton's
//          beam frame, binned from t_min / v_min in steps dt / dv; protons
//          outside the bins are removed;
//   test:  q in {WEPL, theta_out - theta_in, psi_out - psi_in}; per bin the
//          mean mu and the population standard deviation sigma (two passes);
//          keep when |q - mu| <= k_sigma sigma for all three.
//
// One thread per proton, FP64 throughout (the decisions are integer results
// decided by floating point, taken in FP64 as the oracle takes them); the
// per-bin sums are FP64 atomics (their order is not fixed, so a proton within
// rounding of a cut may be decided either way).  The library is compiled
// without implicit multiply-add contraction, so the products and sums below
// round as written.
#include "pct_bins.cuh"
#include "pct_internal.h"

namespace pct {

namespace {

constexpr int kCleanCta = 256;

__device__ __forceinline__ void clean_q(const float* __restrict__ h, int64_t stride, int64_t i, double q[3])
{
    q[0] = (double)h[H_WEPL * stride + i];
    q[1] = (double)h[H_THO * stride + i] - (double)h[H_THI * stride + i];
    q[2] = (double)h[H_PSO * stride + i] - (double)h[H_PSI * stride + i];
}

// pass 1: bin of every proton, bin counts and sums
__global__ void __launch_bounds__(kCleanCta)
k_clean_sum(CleanBins P, const float* __restrict__ h, int64_t stride, int64_t n, int* __restrict__ bin,
            unsigned* __restrict__ cnt, double* __restrict__ sum)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int b = proton_bin(P.bins, h[H_INX * stride + i], h[H_INY * stride + i], h[H_INZ * stride + i],
                            h[H_OUTX * stride + i], h[H_OUTY * stride + i], h[H_OUTZ * stride + i],
                            h[H_PHI * stride + i]);
    bin[i] = b;
    if (b < 0) return;
    double q[3];
    clean_q(h, stride, i, q);
    atomicAdd(cnt + b, 1u);
#pragma unroll
    for (int k = 0; k < 3; ++k) atomicAdd(sum + 3 * (int64_t)b + k, q[k]);
}

// pass 2: sums of squared deviations from the bin means
__global__ void __launch_bounds__(kCleanCta)
k_clean_dev(const float* __restrict__ h, int64_t stride, int64_t n, const int* __restrict__ bin,
            const unsigned* __restrict__ cnt, const double* __restrict__ sum, double* __restrict__ dev2)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int b = bin[i];
    if (b < 0) return;
    double q[3];
    clean_q(h, stride, i, q);
    const double c = (double)cnt[b];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const double d = q[k] - sum[3 * (int64_t)b + k] / c;
        atomicAdd(dev2 + 3 * (int64_t)b + k, d * d);
    }
}

// pass 3: the keep decision
__global__ void __launch_bounds__(kCleanCta)
k_clean_keep(const float* __restrict__ h, int64_t stride, int64_t n, double k_sigma,
             const int* __restrict__ bin, const unsigned* __restrict__ cnt, const double* __restrict__ sum,
             const double* __restrict__ dev2, uint8_t* __restrict__ keep)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int b = bin[i];
    bool k_ok = b >= 0;
    if (k_ok) {
        double q[3];
        clean_q(h, stride, i, q);
        const double c = (double)cnt[b];
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const double mu = sum[3 * (int64_t)b + k] / c;
            const double sigma = sqrt(dev2[3 * (int64_t)b + k] / c);
            k_ok = k_ok && fabs(q[k] - mu) <= k_sigma * sigma;
        }
    }
    keep[i] = k_ok ? 1 : 0;
}

// Order-preserving compaction of the kept protons: per chunk of kChunk
// protons, count; exclusive scan of the chunk counts (one CTA); write each kept
// proton's 12 columns at its position.
constexpr int kChunk = 4096;
constexpr int kScanCta = 1024;

__global__ void __launch_bounds__(kCleanCta)
k_keep_count(const uint8_t* __restrict__ keep, int64_t n, int64_t* __restrict__ chunk)
{
    __shared__ int part[kCleanCta / 32];
    const int64_t base = blockIdx.x * (int64_t)kChunk;
    int c = 0;
    for (int r = threadIdx.x; r < kChunk; r += kCleanCta) {
        const int64_t i = base + r;
        c += (i < n && keep[i]) ? 1 : 0;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
    if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = c;
    __syncthreads();
    if (threadIdx.x == 0) {
        int64_t t = 0;
        for (int w = 0; w < kCleanCta / 32; ++w) t += part[w];
        chunk[blockIdx.x] = t;
    }
}

__global__ void __launch_bounds__(kScanCta)
k_keep_scan(int64_t* __restrict__ chunk, int64_t nchunks, int64_t* __restrict__ total)
{
    __shared__ int64_t part[kScanCta];
    const int64_t per = (nchunks + kScanCta - 1) / kScanCta;
    const int64_t a = threadIdx.x * per, b = a + per < nchunks ? a + per : nchunks;
    int64_t s = 0;
    for (int64_t c = a; c < b; ++c) s += chunk[c];
    part[threadIdx.x] = s;
    __syncthreads();
    for (int o = 1; o < kScanCta; o <<= 1) {
        const int64_t v = threadIdx.x >= o ? part[threadIdx.x - o] : 0;
        __syncthreads();
        part[threadIdx.x] += v;
        __syncthreads();
    }
    int64_t run = part[threadIdx.x] - s;
    for (int64_t c = a; c < b; ++c) {
        const int64_t v = chunk[c];
        chunk[c] = run;
        run += v;
    }
    if (threadIdx.x == kScanCta - 1) *total = part[threadIdx.x];
}

// ncols columns of `stride` floats are copied; column shift_col (if >= 0) gets
// `shift` added on the way
__global__ void __launch_bounds__(kCleanCta)
k_keep_fill(const uint8_t* __restrict__ keep, int64_t n, const int64_t* __restrict__ chunk,
            const float* __restrict__ h, int64_t stride, int ncols, int shift_col, float shift,
            float* __restrict__ out, int64_t out_stride)
{
    __shared__ int part[kCleanCta / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t base = blockIdx.x * (int64_t)kChunk;
    int64_t run = chunk[blockIdx.x];
    for (int r = 0; r < kChunk; r += kCleanCta) {
        const int64_t i = base + r + threadIdx.x;
        const bool v = i < n && keep[i];
        const unsigned bal = __ballot_sync(0xffffffffu, v);
        if (lane == 0) part[warp] = __popc(bal);
        __syncthreads();
        int before = 0, total = 0;
        for (int w = 0; w < kCleanCta / 32; ++w) {
            before += w < warp ? part[w] : 0;
            total += part[w];
        }
        if (v) {
            const int64_t pos = run + before + __popc(bal & ((1u << lane) - 1u));
            for (int f = 0; f < ncols; ++f) {
                const float v = h[f * stride + i];
                out[f * out_stride + pos] = f == shift_col ? v + shift : v;
            }
        }
        run += total;
        __syncthreads();
    }
}

}  // namespace

int64_t clean_chunks(int64_t n)
{
    return (n + kChunk - 1) / kChunk;
}

cudaError_t launch_clean(const Launch& L, const CleanBins& P, const float* hist, int64_t stride, int64_t n,
                         int* bin, unsigned* cnt, double* sum, double* dev2, uint8_t* keep)
{
    if (n <= 0) return cudaSuccess;
    const int64_t nb = (int64_t)P.bins.n_angle * P.bins.n_t * P.bins.n_v;
    cudaError_t e = cudaMemsetAsync(cnt, 0, (size_t)nb * sizeof(unsigned), L.stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(sum, 0, (size_t)nb * 3 * sizeof(double), L.stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(dev2, 0, (size_t)nb * 3 * sizeof(double), L.stream);
    if (e != cudaSuccess) return e;
    const unsigned g = (unsigned)((n + kCleanCta - 1) / kCleanCta);
    k_clean_sum<<<g, kCleanCta, 0, L.stream>>>(P, hist, stride, n, bin, cnt, sum);
    k_clean_dev<<<g, kCleanCta, 0, L.stream>>>(hist, stride, n, bin, cnt, sum, dev2);
    k_clean_keep<<<g, kCleanCta, 0, L.stream>>>(hist, stride, n, P.k_sigma, bin, cnt, sum, dev2, keep);
    *L.launches += 3;
    return cudaGetLastError();
}

cudaError_t launch_flag_count(const Launch& L, const uint8_t* flag, int64_t n, int64_t* chunk, int64_t* total)
{
    if (n <= 0) return cudaMemsetAsync(total, 0, sizeof(int64_t), L.stream);
    const int64_t nc = clean_chunks(n);
    k_keep_count<<<(unsigned)nc, kCleanCta, 0, L.stream>>>(flag, n, chunk);
    k_keep_scan<<<1, kScanCta, 0, L.stream>>>(chunk, nc, total);
    *L.launches += 2;
    return cudaGetLastError();
}

cudaError_t launch_flag_fill(const Launch& L, const uint8_t* flag, int64_t n, const int64_t* chunk,
                             const float* src, int64_t stride, int ncols, int shift_col, float shift, float* out,
                             int64_t out_stride)
{
    if (n <= 0) return cudaSuccess;
    k_keep_fill<<<(unsigned)clean_chunks(n), kCleanCta, 0, L.stream>>>(flag, n, chunk, src, stride, ncols,
                                                                      shift_col, shift, out, out_stride);
    ++*L.launches;
    return cudaGetLastError();
}

cudaError_t launch_flag_compact(const Launch& L, const uint8_t* flag, int64_t n, int64_t* chunk,
                                int64_t* total, const float* src, int64_t stride, int ncols, int shift_col,
                                float shift, float* out, int64_t out_stride)
{
    cudaError_t e = launch_flag_count(L, flag, n, chunk, total);
    if (e == cudaSuccess) e = launch_flag_fill(L, flag, n, chunk, src, stride, ncols, shift_col, shift, out, out_stride);
    return e;
}

cudaError_t launch_keep_compact(const Launch& L, const uint8_t* keep, int64_t n, int64_t* chunk,
                                int64_t* total, const float* hist, int64_t stride, float* out,
                                int64_t out_stride)
{
    return launch_flag_compact(L, keep, n, chunk, total, hist, stride, H_NF, -1, 0.f, out, out_stride);
}

}  // namespace pct
