// pct_peaks.cu -- microbenchmarks that measure the two ceilings of the fused
// DROP block step on the GPU it runs on: FP32 fused multiply-add throughput
// (the MLP and walk arithmetic) and the throughput of float2 atomic adds to
// random addresses of an L2-resident array (the DROP scatter).  They are the
// roofline denominators the benchmark reports against; neither is part of the
// reconstruction.
#include <cuda_runtime.h>

#include "pct.h"

namespace {

constexpr int kFmaChains = 8;     // independent FMA chains per thread (hides the FMA latency)
constexpr int kFmaCta = 256;

__global__ void __launch_bounds__(kFmaCta)
k_fma_loop(float* out, int iters, float a, float b)
{
    float v[kFmaChains];
#pragma unroll
    for (int c = 0; c < kFmaChains; ++c) v[c] = (float)(threadIdx.x + c) * 1e-3f;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int r = 0; r < 16; ++r)
#pragma unroll
            for (int c = 0; c < kFmaChains; ++c) v[c] = fmaf(v[c], a, b);
    }
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < kFmaChains; ++c) s += v[c];
    if (s == 12345.678f) out[0] = s;   // never true for these inputs; keeps the loop live
}

// splitmix64 finaliser (Steele, Lea, Flood 2014): a counter-based hash that
// spreads thread x iteration over the array
__device__ __forceinline__ unsigned long long mix64(unsigned long long z)
{
    z += 0x9e3779b97f4a7c15ull;
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
    return z ^ (z >> 31);
}

__global__ void k_atomic_random(float2* acc, unsigned long long n_slots, int iters, unsigned long long seed)
{
    const unsigned long long t = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x;
    unsigned long long h = mix64(seed ^ (t * 0x2545f4914f6cdd1dull));
    for (int it = 0; it < iters; ++it) {
        h = mix64(h);
        atomicAdd(acc + (h % n_slots), make_float2(1e-3f, 1.f));
    }
}

struct Timer {
    cudaEvent_t a = nullptr, b = nullptr;
    Timer()
    {
        cudaEventCreate(&a);
        cudaEventCreate(&b);
    }
    ~Timer()
    {
        if (a) cudaEventDestroy(a);
        if (b) cudaEventDestroy(b);
    }
};

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

pct_status cuda_status(cudaError_t e)
{
    if (e == cudaSuccess) return PCT_OK;
    cudaGetLastError();
    return PCT_ERR_CUDA;
}

}  // namespace

extern "C" pct_status pct_peak_fp32(int device, int32_t repeats, double* tflops, double* best_ms)
{
    if (!tflops || repeats < 1) return PCT_ERR_ARG;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
        cudaGetLastError();
        return PCT_ERR_ARG;
    }
    DeviceGuard dg(device);
    int sms = 0, per_sm = 0;
    cudaError_t e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
    if (e == cudaSuccess)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_fma_loop, kFmaCta, 0);
    if (e != cudaSuccess) return cuda_status(e);
    float* out = nullptr;
    if ((e = cudaMalloc(&out, sizeof(float))) != cudaSuccess) return cuda_status(e);
    const int iters = 4096;
    const unsigned grid = (unsigned)(sms * per_sm);
    Timer T;
    float best = 1e30f;
    k_fma_loop<<<grid, kFmaCta>>>(out, iters / 16, 0.999f, 1e-4f);   // warm-up
    for (int r = 0; r < repeats && e == cudaSuccess; ++r) {
        cudaEventRecord(T.a);
        k_fma_loop<<<grid, kFmaCta>>>(out, iters, 0.999f, 1e-4f);
        cudaEventRecord(T.b);
        e = cudaEventSynchronize(T.b);
        float ms = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, T.a, T.b);
        if (ms < best) best = ms;
    }
    if (e == cudaSuccess) e = cudaGetLastError();
    cudaFree(out);
    if (e != cudaSuccess) return cuda_status(e);
    const double flops = 2.0 * kFmaChains * 16.0 * iters * (double)grid * kFmaCta;
    *tflops = flops / (best * 1e-3) / 1e12;
    if (best_ms) *best_ms = best;
    return PCT_OK;
}

extern "C" pct_status pct_peak_atomic(int device, int64_t n_slots, int32_t repeats, double* gatomics,
                                      double* best_ms)
{
    if (!gatomics || repeats < 1 || n_slots < 1 || n_slots > ((int64_t)1 << 31)) return PCT_ERR_ARG;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
        cudaGetLastError();
        return PCT_ERR_ARG;
    }
    DeviceGuard dg(device);
    int sms = 0;
    cudaError_t e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
    if (e != cudaSuccess) return cuda_status(e);
    float2* acc = nullptr;
    if ((e = cudaMalloc(&acc, (size_t)n_slots * sizeof(float2))) != cudaSuccess) return cuda_status(e);
    e = cudaMemset(acc, 0, (size_t)n_slots * sizeof(float2));
    const int cta = 256, iters = 2048;
    const unsigned grid = (unsigned)sms * 8u;
    Timer T;
    float best = 1e30f;
    if (e == cudaSuccess) k_atomic_random<<<grid, cta>>>(acc, (unsigned long long)n_slots, iters, 1ull);
    for (int r = 0; r < repeats && e == cudaSuccess; ++r) {
        cudaEventRecord(T.a);
        k_atomic_random<<<grid, cta>>>(acc, (unsigned long long)n_slots, iters, 2ull + r);
        cudaEventRecord(T.b);
        e = cudaEventSynchronize(T.b);
        float ms = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, T.a, T.b);
        if (ms < best) best = ms;
    }
    if (e == cudaSuccess) e = cudaGetLastError();
    cudaFree(acc);
    if (e != cudaSuccess) return cuda_status(e);
    *gatomics = (double)grid * cta * iters / (best * 1e-3) / 1e9;
    if (best_ms) *best_ms = best;
    return PCT_OK;
}
