// pct_batch.h -- private: one scan of a batched DROP launch (pct_batch.cu).
#pragma once

#include "pct_internal.h"

namespace pct {

struct ScanDesc {
    GridC g;
    MlpC mc;
    const uint8_t* mask;
    const float* rec;     // prepared records
    int64_t stride;
    int64_t n;            // protons
    float* x;             // iterate (device, n_vox)
    float2* acc;          // DROP accumulator (device, n_vox, zero on entry)
    int64_t n_vox;
    int iters;
    float lambda;
    int64_t block;
    int cta0, ncta;       // CTA range of the scan
    unsigned* bar;        // barrier arrival counter (zero on entry)
    int* abort;           // set when a barrier wait of the scan gave up (zero on entry)
    unsigned long long* next;   // work counter of the scan's block steps (zero on entry)
};

// lanes: lanes per proton, 32 or 16 (two protons per warp)
size_t batch_smem(int cta);
cudaError_t batch_max_ctas(int cta, int lanes, int device, int* out);
cudaError_t launch_drop_batch(const Launch& L, const ScanDesc* scans_dev, int nscan, int total_ctas,
                              int cta, int lanes, unsigned* flags, int spin_limit, int test_unreachable);

}  // namespace pct
