// pct_api.cu -- the C ABI of libpct (declared in include/pct.h): context
// lifetime, device memory, history upload, and the host-side loops that drive
// the kernels of pct_kernels.cu.  No call aborts or throws across the ABI.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <unordered_map>
#include <vector>

#include "pct.h"
#include "pct_batch.h"
#include "pct_internal.h"

using namespace pct;

namespace pct {

const double kCoef200[6] = {7.457e-6, 4.548e-7, -5.777e-8, 1.301e-8, -9.228e-10, 2.687e-11};

// Sigma(0, w), w = k du in cm: moments int_0^w (w-u)^n f(u) du of the depth
// polynomial f, via int_0^w (w-u)^n u^k du = w^(n+k+1) n! k! / (n+k+1)!, times
// the Highland prefactor E0^2 (1 + 0.038 ln(w/X0))^2 / X0.
void mlp_sigma_table(double du_mm, int kmax, float4* tab)
{
    static const double fact[10] = {1, 1, 2, 6, 24, 120, 720, 5040, 40320, 362880};
    tab[0] = make_float4(0.f, 0.f, 0.f, 0.f);
    for (int k = 1; k <= kmax; ++k) {
        const double w = k * du_mm * 0.1;
        double mom[3] = {0.0, 0.0, 0.0};
        for (int n = 0; n < 3; ++n)
            for (int p = 0; p < 6; ++p)
                mom[n] += kCoef200[p] * std::pow(w, n + p + 1) * fact[n] * fact[p] / fact[n + p + 1];
        const double lf = 1.0 + 0.038 * std::log(w / (double)kX0);
        const double pre = (double)kE0 * (double)kE0 * lf * lf / (double)kX0;
        tab[k] = make_float4((float)(pre * mom[2]), (float)(pre * mom[1]), (float)(pre * mom[0]),
                             (float)(2.0 * pre * mom[1]));
    }
}

}  // namespace pct

namespace {

thread_local std::string g_create_error;

}  // namespace

struct pct_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    pct_grid grid{};
    GridC gc{};
    int64_t n_vox = 0;
    int64_t n_hull = 0;
    uint8_t* d_mask = nullptr;
    uint8_t* d_dist = nullptr;   // chessboard distance to the hull (hull search skipping)
    float4* d_sig1 = nullptr;
    int kmax = 0;
    int kmax_floor = 0;                  // MLP table covers at least this many samples (region sub-contexts)
    int64_t du_um = 0;
    unsigned* d_flags = nullptr;
    unsigned long long* d_next = nullptr;   // work counter of the warp-per-proton kernels
    unsigned long long* d_fallbacks = nullptr;   // protons the round walk passed to the lane walk
    bool loaded = false;                 // pct_load_histories has succeeded once
    bool rec_valid = false;              // the records match the loaded histories and MLP step
    int64_t n = 0, stride = 0, cap = 0;  // protons, column stride, column capacity
    float* d_hist = nullptr;
    float* d_rec = nullptr;
    float2* d_acc = nullptr;
    // lists of the protons with a hull path per DROP block (fused solve)
    int64_t* d_vidx = nullptr;
    int64_t* d_boff = nullptr;
    int64_t* d_chunk = nullptr;
    int64_t vidx_cap = 0, boff_cap = 0, chunk_cap = 0;
    float* d_xtmp = nullptr;
    // stored rows (PCT_MODE_CSR / PCT_MODE_PACKED)
    int mode = PCT_MODE_FUSED;
    int rows_mode = -1;                  // mode the stored rows were built for (-1: none)
    int64_t nnz = 0;
    int64_t* d_rowptr = nullptr;
    int32_t* d_idx = nullptr;
    float* d_len = nullptr;
    uint8_t* d_codes = nullptr;
    uint16_t* d_lens16 = nullptr;
    int chord_code = PCT_CHORD_FIXED16;    // packed chords: fixed point or FP16
    short4* d_start = nullptr;
    int cta = 256;
    int timing = 0;
    int64_t mem_cap = 0;
    int64_t mem_used = 0;
    std::unordered_map<void*, size_t> sizes;
    int64_t launches = 0;
    int64_t fused_launches = 0;
    // batched solve (pct_solve_batch with this context first)
    int graph = 0, autotune = 0, test_unreachable = 0;
    int64_t spin_limit = 1 << 27;
    int batch_cta = 0, batch_ctas = 0, batch_lanes = 32;
    int lanes_opt = 32;                  // lanes per proton of batched solves (PCT_OPT_BATCH_LANES)
    int64_t persist_max = 0;             // pct_solve: persistent launch up to this block size (PCT_OPT_PERSISTENT_BLOCK)
    int walk = kWalkLanes;               // walk of the DROP step and the row writer (PCT_OPT_WALK)
    int64_t graph_replays = 0;
    ScanDesc* d_scans = nullptr;
    unsigned* d_bar = nullptr;
    int* d_abort = nullptr;
    unsigned long long* d_bnext = nullptr;   // per-scan work counters
    int scan_cap = 0;
    cudaStream_t batch_stream = nullptr;
    // uploads from host memory: copy stream and one event per uploaded chunk
    cudaStream_t copy_stream = nullptr;
    cudaEvent_t copy_ready = nullptr;
    std::vector<cudaEvent_t> chunk_ev;
    cudaEvent_t batch_ev[2] = {nullptr, nullptr};
    cudaGraphExec_t graph_exec = nullptr;
    std::vector<int64_t> graph_key;
    // pct_solve: one iteration of block launches captured in a CUDA graph
    int64_t solve_graph_min = 64;        // fewest blocks per iteration to capture (PCT_OPT_SOLVE_GRAPH; 0 = never)
    uint64_t gen = 0;                    // bumped by every change of a kernel argument (allocations, options, loads)
    cudaGraphExec_t solve_exec = nullptr;
    std::vector<int64_t> solve_key;
    int64_t solve_launches = 0;          // launches of one captured iteration
    int64_t solve_replays = 0;
    std::vector<std::vector<int64_t>> tuned_keys;
    std::vector<int> tuned_cta, tuned_lanes;
    std::vector<cudaEvent_t> ev;   // pairs (start, stop) of timed fused launches
    size_t ev_used = 0;
    std::string err;
};

namespace {

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

pct_status fail(pct_ctx* c, pct_status s, const std::string& msg)
{
    if (c) c->err = msg;
    return s;
}

pct_status cuda_fail(pct_ctx* c, cudaError_t e, const char* where)
{
    std::string m = std::string(where) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")";
    return fail(c, e == cudaErrorMemoryAllocation ? PCT_ERR_OOM : PCT_ERR_CUDA, m);
}

pct_status dalloc(pct_ctx* c, void** p, size_t bytes, const char* what)
{
    *p = nullptr;
    ++c->gen;
    if (bytes == 0) bytes = 16;
    if (c->mem_cap > 0 && c->mem_used + (int64_t)bytes > c->mem_cap)
        return fail(c, PCT_ERR_OOM, std::string(what) + ": device memory cap exceeded");
    cudaError_t e = cudaMalloc(p, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
        return fail(c, PCT_ERR_OOM, std::string(what) + ": cudaMalloc failed (" + cudaGetErrorString(e) + ")");
    }
    c->sizes[*p] = bytes;
    c->mem_used += (int64_t)bytes;
    return PCT_OK;
}

void dfree(pct_ctx* c, void* p)
{
    if (!p) return;
    ++c->gen;
    auto it = c->sizes.find(p);
    if (it != c->sizes.end()) {
        c->mem_used -= (int64_t)it->second;
        c->sizes.erase(it);
    }
    cudaFree(p);
}

double step_mm(const pct_ctx* c)
{
    return c->du_um > 0 ? (double)c->du_um * 1e-3
                        : (double)std::fmin(c->grid.dx, std::fmin(c->grid.dy, c->grid.dz));
}

pct_status build_sigma_table(pct_ctx* c)
{
    const double du = step_mm(c);
    const double diag = std::sqrt(std::pow((double)c->grid.nx * c->grid.dx, 2) +
                                  std::pow((double)c->grid.ny * c->grid.dy, 2) +
                                  std::pow((double)c->grid.nz * c->grid.dz, 2));
    const int kmax = std::max((int)std::ceil(diag / du) + 3, c->kmax_floor);
    if (kmax > (1 << 22)) return fail(c, PCT_ERR_ARG, "MLP step too small for this grid");
    std::vector<float4> tab((size_t)kmax + 1);
    mlp_sigma_table(du, kmax, tab.data());
    void* p = nullptr;
    pct_status s = dalloc(c, &p, tab.size() * sizeof(float4), "MLP table");
    if (s != PCT_OK) return s;
    cudaError_t e = cudaMemcpy(p, tab.data(), tab.size() * sizeof(float4), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        dfree(c, p);
        return cuda_fail(c, e, "MLP table upload");
    }
    dfree(c, c->d_sig1);
    c->d_sig1 = (float4*)p;
    c->kmax = kmax;
    return PCT_OK;
}

Geo geo_of(const pct_ctx* c)
{
    Geo G;
    G.g = c->gc;
    const double du = step_mm(c);
    G.mc.du_mm = (float)du;
    G.mc.du_cm = (float)(0.1 * du);
    G.mc.dend_mm = (float)(1e-3 * du);
    for (int k = 0; k < 6; ++k) G.mc.coef[k] = (float)kCoef200[k];
    G.mc.sig1 = c->d_sig1;
    G.mc.kmax = c->kmax;
    // a lane range of cmin segments is deeper than the longest chord of a voxel
    const double diag = std::sqrt((double)c->grid.dx * c->grid.dx + (double)c->grid.dy * c->grid.dy +
                                  (double)c->grid.dz * c->grid.dz);
    G.mc.cmin = (int)std::floor(diag / du) + 1;
    G.mask = c->d_mask;
    G.dist = c->d_dist;
    G.flags = c->d_flags;
    G.walk = c->walk;
    G.fallbacks = c->d_fallbacks;
    return G;
}

Launch launch_of(pct_ctx* c)
{
    return Launch{c->stream, c->cta, &c->launches};
}

pct_status need_histories(pct_ctx* c)
{
    if (!c->loaded) return fail(c, PCT_ERR_STATE, "no proton histories loaded");
    return PCT_OK;
}

// Protons per chunk of an upload from host memory.
constexpr int64_t kUploadChunk = 1 << 22;

// Per-proton records (hull entry/exit, beam frame, FP64-evaluated states):
// computed once per loaded history set and MLP step, kept until either changes.
pct_status prepare(pct_ctx* c)
{
    if (c->n == 0 || c->rec_valid) return PCT_OK;
    cudaError_t e = launch_prepare(launch_of(c), geo_of(c), c->d_hist, c->stride, c->n, c->d_rec);
    if (e != cudaSuccess) return cuda_fail(c, e, "prepare kernel");
    c->rec_valid = true;
    return PCT_OK;
}

pct_status ensure_acc(pct_ctx* c)
{
    if (c->d_acc) return PCT_OK;
    void* p = nullptr;
    pct_status s = dalloc(c, &p, (size_t)c->n_vox * sizeof(float2), "DROP accumulator");
    if (s != PCT_OK) return s;
    c->d_acc = (float2*)p;
    return PCT_OK;
}

pct_status ensure_i64(pct_ctx* c, int64_t** p, int64_t* cap, int64_t need, const char* what)
{
    if (*p && *cap >= need) return PCT_OK;
    dfree(c, *p);
    *p = nullptr;
    *cap = 0;
    void* q = nullptr;
    pct_status s = dalloc(c, &q, (size_t)need * sizeof(int64_t), what);
    if (s != PCT_OK) return s;
    *p = (int64_t*)q;
    *cap = need;
    return PCT_OK;
}

// Valid-proton lists of the DROP blocks of size B (after prepare).
pct_status compact(pct_ctx* c, int64_t B)
{
    pct_status s;
    if ((s = ensure_i64(c, &c->d_vidx, &c->vidx_cap, c->n, "valid-proton list")) != PCT_OK ||
        (s = ensure_i64(c, &c->d_boff, &c->boff_cap, (c->n + B - 1) / B + 1, "block offsets")) != PCT_OK ||
        (s = ensure_i64(c, &c->d_chunk, &c->chunk_cap, compact_chunks(c->n), "compaction scratch")) != PCT_OK)
        return s;
    cudaError_t e = launch_compact(launch_of(c), c->d_rec, c->stride, c->n, B, c->d_chunk, c->d_vidx, c->d_boff);
    return e == cudaSuccess ? PCT_OK : cuda_fail(c, e, "valid-proton lists");
}

// Unit of the packed rows' 16-bit fixed-point chords (mm), 0 for FP16 chords.
// A run's chord lies in one voxel: up to the voxel diagonal, a little more
// where the polyline bends inside the voxel; 1.25 diagonals span the code.
float chord_unit(const pct_ctx* c)
{
    if (c->chord_code != PCT_CHORD_FIXED16) return 0.f;
    const double diag = std::sqrt((double)c->grid.dx * c->grid.dx + (double)c->grid.dy * c->grid.dy +
                                  (double)c->grid.dz * c->grid.dz);
    return (float)(1.25 * diag / 65535.0);
}

int64_t row_bytes(const pct_ctx* c)
{
    int64_t b = 0;
    for (void* p : {(void*)c->d_rowptr, (void*)c->d_idx, (void*)c->d_len, (void*)c->d_codes,
                    (void*)c->d_lens16, (void*)c->d_start}) {
        auto it = c->sizes.find(p);
        if (p && it != c->sizes.end()) b += (int64_t)it->second;
    }
    return b;
}

void drop_rows(pct_ctx* c)
{
    if (c->rows_mode >= 0 && c->stream) cudaStreamSynchronize(c->stream);
    dfree(c, c->d_rowptr);
    dfree(c, c->d_idx);
    dfree(c, c->d_len);
    dfree(c, c->d_codes);
    dfree(c, c->d_lens16);
    dfree(c, c->d_start);
    c->d_rowptr = nullptr;
    c->d_idx = nullptr;
    c->d_len = nullptr;
    c->d_codes = nullptr;
    c->d_lens16 = nullptr;
    c->d_start = nullptr;
    c->nnz = 0;
    c->rows_mode = -1;
}

// Build the stored rows of the current mode: count entries per row, scan to
// row offsets, allocate, fill.  Synchronizes once (to size the entry arrays).
pct_status build_rows(pct_ctx* c)
{
    drop_rows(c);
    if (c->mode == PCT_MODE_FUSED) return PCT_OK;
    const int64_t m = c->n;
    const Launch L = launch_of(c);
    const Geo G = geo_of(c);
    pct_status s = prepare(c);
    if (s != PCT_OK) return s;
    void *p_cnt = nullptr, *p_chunk = nullptr, *p = nullptr;
    if ((s = dalloc(c, &p_cnt, (size_t)(m > 0 ? m : 1) * sizeof(int32_t), "row counts")) != PCT_OK) return s;
    if ((s = dalloc(c, &p_chunk, (size_t)(scan_chunks(m) + 1) * sizeof(int64_t), "scan chunks")) != PCT_OK) {
        dfree(c, p_cnt);
        return s;
    }
    auto cleanup = [&]() {
        dfree(c, p_cnt);
        dfree(c, p_chunk);
    };
    if ((s = dalloc(c, &p, (size_t)(m + 1) * sizeof(int64_t), "row offsets")) != PCT_OK) {
        cleanup();
        return s;
    }
    c->d_rowptr = (int64_t*)p;
    cudaError_t e;
    if (c->mode == PCT_MODE_PACKED) {
        if ((s = dalloc(c, &p, (size_t)(m > 0 ? m : 1) * sizeof(short4), "row starts")) != PCT_OK) {
            cleanup();
            drop_rows(c);
            return s;
        }
        c->d_start = (short4*)p;
        e = launch_pack_count(L, G, c->d_rec, c->stride, m, (int32_t*)p_cnt, c->d_start);
    } else {
        e = launch_csr_count(L, G, c->d_rec, c->stride, m, (int32_t*)p_cnt);
    }
    if (e == cudaSuccess) e = launch_row_scan(L, (const int32_t*)p_cnt, m, c->d_rowptr, (int64_t*)p_chunk);
    int64_t nnz = 0;
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(&nnz, c->d_rowptr + m, sizeof nnz, cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    cleanup();
    if (e != cudaSuccess) {
        drop_rows(c);
        return cuda_fail(c, e, "row count");
    }
    // a row holds at most a few entries per voxel of the grid diagonal
    if (nnz < 0 || nnz > m * (int64_t)(4 * (c->kmax + 8))) {
        drop_rows(c);
        return fail(c, PCT_ERR_DEVICE, "row count out of range (" + std::to_string(nnz) + " entries)");
    }
    const size_t ne = (size_t)(nnz > 0 ? nnz : 1);
    if (c->mode == PCT_MODE_PACKED) {
        if ((s = dalloc(c, &p, ne, "packed row codes")) == PCT_OK) {
            c->d_codes = (uint8_t*)p;
            if ((s = dalloc(c, &p, ne * 2, "packed row chords")) == PCT_OK) c->d_lens16 = (uint16_t*)p;
        }
        if (s == PCT_OK)
            e = launch_pack_fill(L, G, c->d_rec, c->stride, m, c->d_rowptr, c->d_codes, c->d_lens16,
                                 chord_unit(c));
    } else {
        if ((s = dalloc(c, &p, ne * sizeof(int32_t), "CSR indices")) == PCT_OK) {
            c->d_idx = (int32_t*)p;
            if ((s = dalloc(c, &p, ne * sizeof(float), "CSR chords")) == PCT_OK) c->d_len = (float*)p;
        }
        if (s == PCT_OK) e = launch_csr_fill(L, G, c->d_rec, c->stride, m, c->d_rowptr, c->d_idx, c->d_len);
    }
    if (s != PCT_OK) {
        drop_rows(c);
        return s;
    }
    if (e != cudaSuccess) {
        drop_rows(c);
        return cuda_fail(c, e, "row fill");
    }
    c->nnz = nnz;
    c->rows_mode = c->mode;
    return PCT_OK;
}

cudaEvent_t next_event(pct_ctx* c)
{
    if (c->ev_used == c->ev.size()) {
        cudaEvent_t e;
        if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
        c->ev.push_back(e);
    }
    return c->ev[c->ev_used++];
}

}  // namespace

extern "C" {

pct_status pct_create(pct_ctx** out, const pct_grid* grid, const uint8_t* hull_mask, int device,
                      void* cuda_stream)
{
    if (!out || !grid) {
        g_create_error = "pct_create: null argument";
        return PCT_ERR_ARG;
    }
    *out = nullptr;
    const pct_grid& G = *grid;
    if (G.nx < 1 || G.ny < 1 || G.nz < 1 || !(G.dx > 0.f) || !(G.dy > 0.f) || !(G.dz > 0.f) ||
        !std::isfinite(G.dx) || !std::isfinite(G.dy) || !std::isfinite(G.dz) || !std::isfinite(G.ox) ||
        !std::isfinite(G.oy) || !std::isfinite(G.oz)) {
        g_create_error = "pct_create: invalid grid";
        return PCT_ERR_ARG;
    }
    const int64_t n_vox = (int64_t)G.nx * G.ny * G.nz;
    if (n_vox > 0x7fffffffLL) {
        g_create_error = "pct_create: grid over 2^31 voxels";
        return PCT_ERR_ARG;
    }
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
        cudaGetLastError();
        g_create_error = "pct_create: no such CUDA device";
        return PCT_ERR_ARG;
    }
    pct_ctx* c = new (std::nothrow) pct_ctx();
    if (!c) {
        g_create_error = "pct_create: out of host memory";
        return PCT_ERR_OOM;
    }
    DeviceGuard dg(device);
    c->device = device;
    c->grid = G;
    c->n_vox = n_vox;
    c->gc.nx = G.nx;
    c->gc.ny = G.ny;
    c->gc.nz = G.nz;
    c->gc.dx = G.dx;
    c->gc.dy = G.dy;
    c->gc.dz = G.dz;
    c->gc.ox = G.ox;
    c->gc.oy = G.oy;
    c->gc.oz = G.oz;
    c->gc.idx = 1.f / G.dx;
    c->gc.idy = 1.f / G.dy;
    c->gc.idz = 1.f / G.dz;
    pct_status s = PCT_OK;
    cudaError_t e;
    if (cuda_stream) {
        c->stream = (cudaStream_t)cuda_stream;
    } else {
        e = cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking);
        if (e != cudaSuccess) {
            g_create_error = std::string("pct_create: stream: ") + cudaGetErrorString(e);
            delete c;
            return PCT_ERR_CUDA;
        }
        c->own_stream = true;
    }
    std::vector<uint8_t> mask((size_t)n_vox, 1);
    if (hull_mask)
        for (int64_t j = 0; j < n_vox; ++j) mask[(size_t)j] = hull_mask[j] ? 1 : 0;
    for (int64_t j = 0; j < n_vox; ++j) c->n_hull += mask[(size_t)j];
    void* p = nullptr;
    if ((s = dalloc(c, &p, (size_t)n_vox, "hull mask")) == PCT_OK) {
        c->d_mask = (uint8_t*)p;
        e = cudaMemcpy(c->d_mask, mask.data(), (size_t)n_vox, cudaMemcpyHostToDevice);
        if (e != cudaSuccess) s = cuda_fail(c, e, "hull mask upload");
    }
    if (s == PCT_OK && (s = dalloc(c, &p, (size_t)n_vox, "hull distance map")) == PCT_OK) {
        c->d_dist = (uint8_t*)p;
        void* tmp = nullptr;
        if ((s = dalloc(c, &tmp, (size_t)n_vox, "hull distance scratch")) == PCT_OK) {
            e = launch_hull_dist(launch_of(c), c->d_mask, G.nx, G.ny, G.nz, (uint8_t*)tmp, c->d_dist);
            if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
            if (e != cudaSuccess) s = cuda_fail(c, e, "hull distance map");
            dfree(c, tmp);
        }
    }
    if (s == PCT_OK && (s = dalloc(c, &p, sizeof(unsigned), "flags")) == PCT_OK) {
        c->d_flags = (unsigned*)p;
        e = cudaMemset(c->d_flags, 0, sizeof(unsigned));
        if (e != cudaSuccess) s = cuda_fail(c, e, "flags");
    }
    if (s == PCT_OK && (s = dalloc(c, &p, sizeof(unsigned long long), "work counter")) == PCT_OK)
        c->d_next = (unsigned long long*)p;
    if (s == PCT_OK && (s = dalloc(c, &p, sizeof(unsigned long long), "walk fallback counter")) == PCT_OK) {
        c->d_fallbacks = (unsigned long long*)p;
        e = cudaMemset(p, 0, sizeof(unsigned long long));
        if (e != cudaSuccess) s = cuda_fail(c, e, "walk fallback counter");
    }
    if (s == PCT_OK) s = build_sigma_table(c);
    if (s != PCT_OK) {
        g_create_error = "pct_create: " + c->err;
        pct_destroy(c);
        return s;
    }
    *out = c;
    return PCT_OK;
}

void pct_destroy(pct_ctx* c)
{
    if (!c) return;
    DeviceGuard dg(c->device);
    if (c->stream) cudaStreamSynchronize(c->stream);
    for (auto& kv : c->sizes) cudaFree(kv.first);
    c->sizes.clear();
    for (cudaEvent_t e : c->ev) cudaEventDestroy(e);
    if (c->graph_exec) cudaGraphExecDestroy(c->graph_exec);
    if (c->solve_exec) cudaGraphExecDestroy(c->solve_exec);
    for (cudaEvent_t e : c->batch_ev)
        if (e) cudaEventDestroy(e);
    if (c->batch_stream) cudaStreamDestroy(c->batch_stream);
    for (cudaEvent_t e : c->chunk_ev)
        if (e) cudaEventDestroy(e);
    if (c->copy_ready) cudaEventDestroy(c->copy_ready);
    if (c->copy_stream) cudaStreamDestroy(c->copy_stream);
    if (c->own_stream && c->stream) cudaStreamDestroy(c->stream);
    delete c;
}

const char* pct_last_error(const pct_ctx* c)
{
    return c ? c->err.c_str() : g_create_error.c_str();
}

pct_status pct_set_option(pct_ctx* c, int32_t key, int64_t value)
{
    if (!c) return PCT_ERR_ARG;
    DeviceGuard dg(c->device);
    ++c->gen;
    switch (key) {
    case PCT_OPT_SOLVE_GRAPH:
        if (value < 0) return fail(c, PCT_ERR_ARG, "solve graph threshold must be >= 0");
        c->solve_graph_min = value;
        return PCT_OK;
    case PCT_OPT_CTA_THREADS:
        if (value < 32 || value > 256 || value % 32) return fail(c, PCT_ERR_ARG, "CTA threads must be 32..256, multiple of 32");
        c->cta = (int)value;
        return PCT_OK;
    case PCT_OPT_MLP_STEP_UM: {
        if (value < 0 || value > 100000) return fail(c, PCT_ERR_ARG, "MLP step out of range");
        drop_rows(c);
        c->rec_valid = false;
        const int64_t old = c->du_um;
        c->du_um = value;
        pct_status s = build_sigma_table(c);
        if (s != PCT_OK) c->du_um = old;
        return s;
    }
    case PCT_OPT_MEM_CAP_BYTES:
        if (value < 0) return fail(c, PCT_ERR_ARG, "negative memory cap");
        c->mem_cap = value;
        return PCT_OK;
    case PCT_OPT_TIMING:
        if (value < 0 || value > 0x7fffffff) return fail(c, PCT_ERR_ARG, "timing period must be >= 0");
        c->timing = (int)value;
        return PCT_OK;
    case PCT_OPT_GRAPH:
        c->graph = value ? 1 : 0;
        return PCT_OK;
    case PCT_OPT_AUTOTUNE:
        c->autotune = value ? 1 : 0;
        return PCT_OK;
    case PCT_OPT_PERSISTENT_BLOCK:
        if (value < 0) return fail(c, PCT_ERR_ARG, "negative persistent block size");
        c->persist_max = value;
        return PCT_OK;
    case PCT_OPT_WALK:
        if (value != PCT_WALK_LANES && value != PCT_WALK_ROUNDS) return fail(c, PCT_ERR_ARG, "unknown walk");
        c->walk = (int)value;
        return PCT_OK;
    case PCT_OPT_BATCH_LANES:
        if (value != 32 && value != 16) return fail(c, PCT_ERR_ARG, "lanes per proton must be 32 or 16");
        c->lanes_opt = (int)value;
        return PCT_OK;
    case PCT_OPT_SPIN_LIMIT:
        if (value < 1 || value > (int64_t)1 << 30) return fail(c, PCT_ERR_ARG, "spin limit must be 1..2^30");
        c->spin_limit = value;
        return PCT_OK;
    case PCT_OPT_TEST_UNREACHABLE_BARRIER:
        c->test_unreachable = value ? 1 : 0;
        return PCT_OK;
    case PCT_OPT_MODE:
        if (value != PCT_MODE_FUSED && value != PCT_MODE_CSR && value != PCT_MODE_PACKED)
            return fail(c, PCT_ERR_ARG, "unknown mode");
        if ((int)value != c->mode) drop_rows(c);
        c->mode = (int)value;
        return PCT_OK;
    case PCT_OPT_CHORD_CODE:
        if (value != PCT_CHORD_FIXED16 && value != PCT_CHORD_FP16) return fail(c, PCT_ERR_ARG, "unknown chord code");
        if ((int)value != c->chord_code && c->mode == PCT_MODE_PACKED) drop_rows(c);
        c->chord_code = (int)value;
        return PCT_OK;
    default:
        return fail(c, PCT_ERR_ARG, "unknown option key");
    }
}

pct_status pct_get_option(const pct_ctx* c, int32_t key, int64_t* value)
{
    if (!c || !value) return PCT_ERR_ARG;
    switch (key) {
    case PCT_OPT_CTA_THREADS: *value = c->cta; return PCT_OK;
    case PCT_OPT_MLP_STEP_UM: *value = (int64_t)std::llround(step_mm(c) * 1000.0); return PCT_OK;
    case PCT_OPT_MEM_CAP_BYTES: *value = c->mem_cap; return PCT_OK;
    case PCT_OPT_TIMING: *value = c->timing; return PCT_OK;
    case PCT_OPT_MODE: *value = c->mode; return PCT_OK;
    case PCT_OPT_CHORD_CODE: *value = c->chord_code; return PCT_OK;
    case PCT_OPT_GRAPH: *value = c->graph; return PCT_OK;
    case PCT_OPT_SOLVE_GRAPH: *value = c->solve_graph_min; return PCT_OK;
    case PCT_OPT_AUTOTUNE: *value = c->autotune; return PCT_OK;
    case PCT_OPT_BATCH_LANES: *value = c->lanes_opt; return PCT_OK;
    case PCT_OPT_WALK: *value = c->walk; return PCT_OK;
    case PCT_OPT_PERSISTENT_BLOCK: *value = c->persist_max; return PCT_OK;
    case PCT_OPT_SPIN_LIMIT: *value = c->spin_limit; return PCT_OK;
    case PCT_OPT_TEST_UNREACHABLE_BARRIER: *value = c->test_unreachable; return PCT_OK;
    default: return PCT_ERR_ARG;
    }
}

pct_status pct_load_histories(pct_ctx* c, int64_t n, const float* const in_xyz[3],
                              const float* const out_xyz[3], const float* const ang_in[2],
                              const float* const ang_out[2], const float* gantry_rad,
                              const float* wepl_mm, int ptrs_on_device)
{
    if (!c) return PCT_ERR_ARG;
    if (n < 0) return fail(c, PCT_ERR_ARG, "negative proton count");
    DeviceGuard dg(c->device);
    ++c->gen;
    drop_rows(c);
    c->rec_valid = false;
    if (n == 0) {
        c->n = 0;
        c->loaded = true;
        return PCT_OK;
    }
    if (!in_xyz || !out_xyz || !ang_in || !ang_out || !gantry_rad || !wepl_mm)
        return fail(c, PCT_ERR_ARG, "null history pointer");
    const float* src[H_NF] = {in_xyz[0], in_xyz[1], in_xyz[2], out_xyz[0], out_xyz[1], out_xyz[2],
                              ang_in[0], ang_in[1], ang_out[0], ang_out[1], gantry_rad, wepl_mm};
    for (int f = 0; f < H_NF; ++f)
        if (!src[f]) return fail(c, PCT_ERR_ARG, "null history pointer");
    const int64_t stride = (n + 31) / 32 * 32;
    if (stride > c->cap) {
        cudaStreamSynchronize(c->stream);
        dfree(c, c->d_hist);
        dfree(c, c->d_rec);
        c->d_hist = c->d_rec = nullptr;
        c->cap = 0;
        c->n = 0;
        c->loaded = false;
        void* p = nullptr;
        pct_status s = dalloc(c, &p, (size_t)stride * H_NF * sizeof(float), "histories");
        if (s != PCT_OK) return s;
        c->d_hist = (float*)p;
        s = dalloc(c, &p, (size_t)stride * R_NF * sizeof(float), "proton records");
        if (s != PCT_OK) {
            dfree(c, c->d_hist);
            c->d_hist = nullptr;
            return s;
        }
        c->d_rec = (float*)p;
        c->cap = stride;
    }
    c->stride = stride;
    if (ptrs_on_device) {
        for (int f = 0; f < H_NF; ++f) {
            cudaError_t e = cudaMemcpyAsync(c->d_hist + (size_t)f * stride, src[f], (size_t)n * sizeof(float),
                                            cudaMemcpyDeviceToDevice, c->stream);
            if (e != cudaSuccess) return cuda_fail(c, e, "history copy");
        }
        c->n = n;
        c->loaded = true;
        return PCT_OK;
    }
    // From host memory: upload in chunks on the copy stream (after the work
    // already on the context stream) and prepare each chunk's records on the
    // context stream as soon as it has landed, so the record kernel runs under
    // the rest of the upload.
    cudaError_t e = cudaSuccess;
    if (!c->copy_stream) e = cudaStreamCreateWithFlags(&c->copy_stream, cudaStreamNonBlocking);
    if (e == cudaSuccess && !c->copy_ready) e = cudaEventCreateWithFlags(&c->copy_ready, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventRecord(c->copy_ready, c->stream);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(c->copy_stream, c->copy_ready, 0);
    if (e != cudaSuccess) return cuda_fail(c, e, "upload stream");
    c->n = n;
    c->loaded = true;
    c->rec_valid = false;
    const int64_t nchunk = (n + kUploadChunk - 1) / kUploadChunk;
    while ((int64_t)c->chunk_ev.size() < nchunk) {
        cudaEvent_t ev = nullptr;
        if ((e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming)) != cudaSuccess)
            return cuda_fail(c, e, "upload events");
        c->chunk_ev.push_back(ev);
    }
    const Launch L = launch_of(c);
    const Geo G = geo_of(c);
    for (int64_t k = 0; k < nchunk && e == cudaSuccess; ++k) {
        const int64_t a = k * kUploadChunk, cnt = std::min(kUploadChunk, n - a);
        for (int f = 0; f < H_NF && e == cudaSuccess; ++f)
            e = cudaMemcpyAsync(c->d_hist + (size_t)f * stride + a, src[f] + a, (size_t)cnt * sizeof(float),
                                cudaMemcpyHostToDevice, c->copy_stream);
        if (e == cudaSuccess) e = cudaEventRecord(c->chunk_ev[(size_t)k], c->copy_stream);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(c->stream, c->chunk_ev[(size_t)k], 0);
        if (e == cudaSuccess) e = launch_prepare_range(L, G, c->d_hist, stride, a, cnt, c->d_rec);
    }
    // the host buffers may be reused once the copies are done
    cudaError_t es = cudaStreamSynchronize(c->copy_stream);
    if (e == cudaSuccess) e = es;
    if (e != cudaSuccess) {
        c->loaded = false;
        c->n = 0;
        return cuda_fail(c, e, "history upload");
    }
    c->rec_valid = true;
    return PCT_OK;
}

pct_status pct_hull_states(pct_ctx* c, int64_t first, int64_t count, float* out)
{
    if (!c) return PCT_ERR_ARG;
    if (first < 0 || count < 0 || first + count > c->n) return fail(c, PCT_ERR_ARG, "proton range out of bounds");
    if (count > 0 && !out) return fail(c, PCT_ERR_ARG, "null output");
    DeviceGuard dg(c->device);
    pct_status s = need_histories(c);
    if (s == PCT_OK) s = prepare(c);
    if (s != PCT_OK) return s;
    cudaError_t e = launch_hull_states(launch_of(c), c->d_rec, c->stride, first, count, out);
    return e == cudaSuccess ? PCT_OK : cuda_fail(c, e, "hull states");
}

pct_status pct_hull_distance(pct_ctx* c, uint8_t* out)
{
    if (!c) return PCT_ERR_ARG;
    if (!out) return fail(c, PCT_ERR_ARG, "null output");
    DeviceGuard dg(c->device);
    cudaError_t e = cudaMemcpyAsync(out, c->d_dist, (size_t)c->n_vox, cudaMemcpyDeviceToDevice, c->stream);
    return e == cudaSuccess ? PCT_OK : cuda_fail(c, e, "hull distance copy");
}

pct_status pct_mlp(pct_ctx* c, int64_t first, int64_t count, int32_t max_pts, float* out_xyz,
                   int32_t* out_npts)
{
    if (!c) return PCT_ERR_ARG;
    if (first < 0 || count < 0 || first + count > c->n) return fail(c, PCT_ERR_ARG, "proton range out of bounds");
    if (max_pts < 2) return fail(c, PCT_ERR_ARG, "max_pts must be >= 2");
    if (count > 0 && (!out_xyz || !out_npts)) return fail(c, PCT_ERR_ARG, "null output");
    DeviceGuard dg(c->device);
    pct_status s = need_histories(c);
    if (s == PCT_OK) s = prepare(c);
    if (s != PCT_OK) return s;
    cudaError_t e = launch_mlp_points(launch_of(c), geo_of(c), c->d_rec, c->stride, first, count,
                                      max_pts, out_xyz, out_npts);
    return e == cudaSuccess ? PCT_OK : cuda_fail(c, e, "MLP kernel");
}

pct_status pct_rows(pct_ctx* c, int64_t first, int64_t count, int32_t max_nnz, int32_t* out_idx,
                    float* out_len, int32_t* out_nnz)
{
    if (!c) return PCT_ERR_ARG;
    if (first < 0 || count < 0 || first + count > c->n) return fail(c, PCT_ERR_ARG, "proton range out of bounds");
    if (max_nnz < 0) return fail(c, PCT_ERR_ARG, "negative max_nnz");
    if (count > 0 && (!out_nnz || (max_nnz > 0 && (!out_idx || !out_len))))
        return fail(c, PCT_ERR_ARG, "null output");
    DeviceGuard dg(c->device);
    pct_status s = need_histories(c);
    if (s == PCT_OK) s = prepare(c);
    if (s != PCT_OK) return s;
    cudaError_t e = launch_rows(launch_of(c), geo_of(c), c->d_rec, c->stride, first, count, max_nnz,
                                out_idx, out_len, out_nnz);
    return e == cudaSuccess ? PCT_OK : cuda_fail(c, e, "row kernel");
}

pct_status pct_forward(pct_ctx* c, const float* x, float* y)
{
    if (!c) return PCT_ERR_ARG;
    if (c->n > 0 && (!x || !y)) return fail(c, PCT_ERR_ARG, "null vector");
    DeviceGuard dg(c->device);
    pct_status s = need_histories(c);
    if (s == PCT_OK) s = prepare(c);
    if (s != PCT_OK) return s;
    cudaError_t e = launch_forward(launch_of(c), geo_of(c), c->d_rec, c->stride, c->n, x, y, c->d_next);
    return e == cudaSuccess ? PCT_OK : cuda_fail(c, e, "forward kernel");
}

pct_status pct_adjoint(pct_ctx* c, const float* y, float* g)
{
    if (!c) return PCT_ERR_ARG;
    if (!g || (c->n > 0 && !y)) return fail(c, PCT_ERR_ARG, "null vector");
    DeviceGuard dg(c->device);
    pct_status s = need_histories(c);
    if (s == PCT_OK) s = prepare(c);
    if (s != PCT_OK) return s;
    cudaError_t e = cudaMemsetAsync(g, 0, (size_t)c->n_vox * sizeof(float), c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "adjoint clear");
    e = launch_adjoint(launch_of(c), geo_of(c), c->d_rec, c->stride, c->n, y, g, c->d_next);
    return e == cudaSuccess ? PCT_OK : cuda_fail(c, e, "adjoint kernel");
}

constexpr int64_t kSolveGraphMaxBlocks = 8192;

// The context's internal stream (batched solves, graph replays of pct_solve) and
// the two events that order it after and before the context's stream.
static pct_status ensure_aux_stream(pct_ctx* c)
{
    if (c->batch_stream) return PCT_OK;
    cudaError_t e = cudaStreamCreateWithFlags(&c->batch_stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->batch_ev[0], cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->batch_ev[1], cudaEventDisableTiming);
    return e == cudaSuccess ? PCT_OK : cuda_fail(c, e, "internal stream");
}

pct_status pct_solve(pct_ctx* c, int32_t iters, float lambda, int64_t block_size, float* x)
{
    if (!c) return PCT_ERR_ARG;
    if (!x) return fail(c, PCT_ERR_ARG, "null x");
    if (iters < 0) return fail(c, PCT_ERR_ARG, "negative iteration count");
    if (block_size < 1) return fail(c, PCT_ERR_ARG, "block size must be >= 1");
    if (!std::isfinite(lambda)) return fail(c, PCT_ERR_ARG, "non-finite lambda");
    DeviceGuard dg(c->device);
    pct_status s = need_histories(c);
    if (s != PCT_OK) return s;
    if (c->n == 0 || iters == 0) return PCT_OK;
    if (c->mode == PCT_MODE_FUSED && c->persist_max > 0 && block_size <= c->persist_max && c->d_hist) {
        // every block step of every iteration in one persistent cooperative
        // launch: the batched solve with this scan alone (no launch per block)
        pct_ctx* cs[1] = {c};
        float* xs[1] = {x};
        return pct_solve_batch(cs, 1, &iters, &lambda, &block_size, xs);
    }
    if ((s = ensure_acc(c)) != PCT_OK) return s;
    if (c->mode == PCT_MODE_FUSED) {
        if ((s = prepare(c)) != PCT_OK) return s;
        if ((s = compact(c, block_size)) != PCT_OK) return s;
    } else if (c->rows_mode != c->mode) {
        if ((s = build_rows(c)) != PCT_OK) return s;
    }
    cudaError_t e = cudaMemsetAsync(c->d_acc, 0, (size_t)c->n_vox * sizeof(float2), c->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->d_next, 0, sizeof(unsigned long long), c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "accumulator clear");
    const Launch L = launch_of(c);
    const Geo G = geo_of(c);
    const float* b = c->d_hist ? c->d_hist + (size_t)H_WEPL * c->stride : nullptr;
    // the block kernel of block `first` and the block apply, with launch shape Lx
    auto block_kernel = [&](const Launch& Lx, int64_t first) -> cudaError_t {
        const int64_t count = block_size < c->n - first ? block_size : c->n - first;
        if (c->mode == PCT_MODE_CSR)
            return launch_drop_csr(Lx, c->d_flags, c->d_rowptr, c->d_idx, c->d_len, b, first, count, x, c->d_acc);
        if (c->mode == PCT_MODE_PACKED)
            return launch_drop_packed(Lx, c->gc, c->d_flags, c->d_rowptr, c->d_start, c->d_codes, c->d_lens16,
                                      chord_unit(c), b, first, count, x, c->d_acc);
        return launch_drop_fused(Lx, G, c->d_rec, c->stride, c->d_vidx, c->d_boff, first / block_size, count, x,
                                 c->d_acc, c->d_next);
    };
    auto apply = [&](const Launch& Lx) -> cudaError_t {
        return launch_drop_apply(Lx, c->n_vox, c->d_mask, x, c->d_acc, lambda, c->d_next);
    };
    const int64_t nblocks = (c->n + block_size - 1) / block_size;
    // capture and instantiation cost ~2.3 us per node: beyond kSolveGraphMaxBlocks blocks per
    // iteration (torso at B = 3200: 36250) it outweighs the launch gaps the replay saves
    if (c->solve_graph_min > 0 && nblocks >= c->solve_graph_min && nblocks <= kSolveGraphMaxBlocks &&
        iters >= 2 && c->timing == 0) {
        if ((s = ensure_aux_stream(c)) != PCT_OK) return s;
        cudaStream_t bs = c->batch_stream;
        int32_t lam_bits;
        std::memcpy(&lam_bits, &lambda, sizeof lam_bits);
        const std::vector<int64_t> key = {(int64_t)c->gen, (int64_t)(uintptr_t)x, block_size, lam_bits, c->n};
        if (!c->solve_exec || c->solve_key != key) {
            if (c->solve_exec) cudaGraphExecDestroy(c->solve_exec);
            c->solve_exec = nullptr;
            const int64_t before = c->launches;
            const Launch Lg{bs, c->cta, &c->launches};
            cudaGraph_t g = nullptr;
            e = cudaStreamBeginCapture(bs, cudaStreamCaptureModeThreadLocal);
            if (e != cudaSuccess) return cuda_fail(c, e, "solve graph capture");
            for (int64_t first = 0; first < c->n && e == cudaSuccess; first += block_size) {
                e = block_kernel(Lg, first);
                if (e == cudaSuccess) e = apply(Lg);
            }
            cudaError_t e2 = cudaStreamEndCapture(bs, &g);
            if (e != cudaSuccess) {
                if (g) cudaGraphDestroy(g);
                c->launches = before;
                return cuda_fail(c, e, "DROP kernels (graph capture)");
            }
            if (e2 != cudaSuccess) return cuda_fail(c, e2, "solve graph capture");
            e = cudaGraphInstantiate(&c->solve_exec, g, 0);
            cudaGraphDestroy(g);
            if (e != cudaSuccess) {
                c->solve_exec = nullptr;
                return cuda_fail(c, e, "solve graph instantiate");
            }
            c->solve_launches = c->launches - before;
            c->launches = before;
            c->solve_key = key;
        }
        e = cudaEventRecord(c->batch_ev[0], c->stream);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(bs, c->batch_ev[0], 0);
        for (int32_t it = 0; it < iters && e == cudaSuccess; ++it) {
            e = cudaGraphLaunch(c->solve_exec, bs);
            if (e == cudaSuccess) {
                ++c->solve_replays;
                c->launches += c->solve_launches;
                c->fused_launches += nblocks;
            }
        }
        if (e == cudaSuccess) e = cudaEventRecord(c->batch_ev[1], bs);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(c->stream, c->batch_ev[1], 0);
        return e == cudaSuccess ? PCT_OK : cuda_fail(c, e, "solve graph launch");
    }
    for (int32_t it = 0; it < iters; ++it) {
        for (int64_t first = 0; first < c->n; first += block_size) {
            cudaEvent_t e0 = nullptr, e1 = nullptr;
            if (c->timing > 0 && c->fused_launches % c->timing == 0) {
                e0 = next_event(c);
                e1 = next_event(c);
                if (e0) cudaEventRecord(e0, c->stream);
            }
            e = block_kernel(L, first);
            if (e != cudaSuccess) return cuda_fail(c, e, "DROP kernel");
            ++c->fused_launches;
            if (e1) cudaEventRecord(e1, c->stream);
            e = apply(L);
            if (e != cudaSuccess) return cuda_fail(c, e, "DROP apply kernel");
        }
    }
    return PCT_OK;
}

pct_status pct_clean(pct_ctx* c, const pct_clean_params* p, uint8_t* keep_out, int64_t* n_kept)
{
    if (!c) return PCT_ERR_ARG;
    if (!p) return fail(c, PCT_ERR_ARG, "null cleaning parameters");
    const int64_t nb = (int64_t)p->n_angle * p->n_t * p->n_v;
    if (p->n_angle < 1 || p->n_t < 1 || p->n_v < 1 || nb > 0x7fffffffLL)
        return fail(c, PCT_ERR_ARG, "bin counts must be >= 1 with fewer than 2^31 bins");
    if (!(p->angle_step > 0.0) || !(p->dt > 0.0) || !(p->dv > 0.0) || !(p->k_sigma >= 0.0) ||
        !std::isfinite(p->angle_step) || !std::isfinite(p->dt) || !std::isfinite(p->dv) ||
        !std::isfinite(p->t_min) || !std::isfinite(p->v_min) || !std::isfinite(p->k_sigma))
        return fail(c, PCT_ERR_ARG, "bin widths must be finite and > 0, k_sigma finite and >= 0");
    DeviceGuard dg(c->device);
    pct_status s = need_histories(c);
    if (s != PCT_OK) return s;
    const int64_t n = c->n;
    if (n == 0) {
        if (n_kept) *n_kept = 0;
        return PCT_OK;
    }
    const CleanBins P{{p->n_angle, p->n_t, p->n_v, p->angle_step, p->t_min, p->dt, p->v_min, p->dv},
                      p->k_sigma};
    void *p_bin = nullptr, *p_cnt = nullptr, *p_sum = nullptr, *p_dev = nullptr, *p_keep = nullptr;
    void *p_chunk = nullptr, *p_total = nullptr, *p_new = nullptr;
    auto cleanup = [&]() {
        for (void* q : {p_bin, p_cnt, p_sum, p_dev, p_keep, p_chunk, p_total}) dfree(c, q);
    };
    if ((s = dalloc(c, &p_bin, (size_t)n * sizeof(int), "cleaning bins")) != PCT_OK ||
        (s = dalloc(c, &p_cnt, (size_t)nb * sizeof(unsigned), "cleaning counts")) != PCT_OK ||
        (s = dalloc(c, &p_sum, (size_t)nb * 3 * sizeof(double), "cleaning sums")) != PCT_OK ||
        (s = dalloc(c, &p_dev, (size_t)nb * 3 * sizeof(double), "cleaning deviations")) != PCT_OK ||
        (!keep_out && (s = dalloc(c, &p_keep, (size_t)n, "keep flags")) != PCT_OK) ||
        (s = dalloc(c, &p_chunk, (size_t)clean_chunks(n) * sizeof(int64_t), "compaction scratch")) != PCT_OK ||
        (s = dalloc(c, &p_total, sizeof(int64_t), "kept count")) != PCT_OK ||
        (s = dalloc(c, &p_new, (size_t)c->cap * H_NF * sizeof(float), "cleaned histories")) != PCT_OK) {
        cleanup();
        return s;
    }
    uint8_t* keep = keep_out ? keep_out : (uint8_t*)p_keep;
    const Launch L = launch_of(c);
    cudaError_t e = launch_clean(L, P, c->d_hist, c->stride, n, (int*)p_bin, (unsigned*)p_cnt, (double*)p_sum,
                                 (double*)p_dev, keep);
    if (e == cudaSuccess)
        e = launch_keep_compact(L, keep, n, (int64_t*)p_chunk, (int64_t*)p_total, c->d_hist, c->stride,
                                (float*)p_new, c->stride);
    int64_t kept = 0;
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(&kept, p_total, sizeof kept, cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    cleanup();
    if (e != cudaSuccess) {
        dfree(c, p_new);
        return cuda_fail(c, e, "data cleaning");
    }
    // the kept protons replace the loaded set (same column stride, which is at
    // least the new count); records and stored rows follow the new set
    drop_rows(c);
    dfree(c, c->d_hist);
    c->d_hist = (float*)p_new;
    c->n = kept;
    c->rec_valid = false;
    if (n_kept) *n_kept = kept;
    return PCT_OK;
}

pct_status pct_solve_regions(pct_ctx* c, int32_t n_regions, int32_t halo, int32_t iters, float lambda,
                             int64_t block_size, float* x, int64_t* region_protons)
{
    if (!c) return PCT_ERR_ARG;
    if (!x) return fail(c, PCT_ERR_ARG, "null x");
    const int nz = c->grid.nz;
    if (n_regions < 1 || n_regions > nz) return fail(c, PCT_ERR_ARG, "regions must be 1..nz");
    if (halo < 0) return fail(c, PCT_ERR_ARG, "negative overlap");
    if (iters < 0 || block_size < 1 || !std::isfinite(lambda))
        return fail(c, PCT_ERR_ARG, "iters < 0, block size < 1 or non-finite lambda");
    DeviceGuard dg(c->device);
    pct_status s = need_histories(c);
    if (s != PCT_OK) return s;
    if ((s = prepare(c)) != PCT_OK) return s;
    const int64_t plane = (int64_t)c->grid.nx * c->grid.ny;
    const Launch L = launch_of(c);
    // 1: setupImageRegions -- core slices [lo, hi), extended by `halo` slices
    struct Region {
        int lo, hi, elo, ehi;
        int64_t count = 0;
        pct_ctx* sub = nullptr;
        float* x = nullptr;
    };
    std::vector<Region> R((size_t)n_regions);
    for (int r = 0; r < n_regions; ++r) {
        Region& g = R[(size_t)r];
        g.lo = (int)((int64_t)r * nz / n_regions);
        g.hi = (int)((int64_t)(r + 1) * nz / n_regions);
        g.elo = std::max(0, g.lo - halo);
        g.ehi = std::min(nz, g.hi + halo);
    }
    std::vector<uint8_t> mask((size_t)c->n_vox);
    cudaError_t e = cudaMemcpyAsync(mask.data(), c->d_mask, (size_t)c->n_vox, cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "hull mask read");
    void *p_flag = nullptr, *p_chunk = nullptr, *p_total = nullptr;
    auto cleanup = [&]() {
        for (Region& g : R)
            if (g.sub) pct_destroy(g.sub);
        dfree(c, p_flag);
        dfree(c, p_chunk);
        dfree(c, p_total);
    };
    const int64_t n = c->n;
    if ((s = dalloc(c, &p_flag, (size_t)std::max<int64_t>(n, 1), "region flags")) != PCT_OK ||
        (s = dalloc(c, &p_chunk, (size_t)std::max<int64_t>(clean_chunks(n), 1) * sizeof(int64_t), "region scan")) != PCT_OK ||
        (s = dalloc(c, &p_total, sizeof(int64_t), "region count")) != PCT_OK) {
        cleanup();
        return s;
    }
    for (Region& g : R) {
        // a sub-context on the region's slab: same voxels, the hull slab, the
        // same MLP spacing and a table as long as the full volume's
        pct_grid sg = c->grid;
        sg.nz = g.ehi - g.elo;
        sg.oz = (float)((double)c->grid.oz + (double)g.elo * (double)c->grid.dz);
        if ((s = pct_create(&g.sub, &sg, mask.data() + (size_t)g.elo * plane, c->device, c->stream)) != PCT_OK) {
            s = fail(c, s, std::string("region context: ") + pct_last_error(nullptr));
            cleanup();
            return s;
        }
        pct_ctx* sub = g.sub;
        sub->cta = c->cta;
        sub->walk = c->walk;
        sub->persist_max = c->persist_max;
        sub->du_um = c->du_um;
        sub->kmax_floor = c->kmax;
        if ((s = build_sigma_table(sub)) != PCT_OK) {
            s = fail(c, s, "region MLP table: " + sub->err);
            cleanup();
            return s;
        }
        // 2: identifyProtonsPassingRegions; 3: allocateMemoryForProtonsPerGPU
        e = launch_region_flags(L, c->d_rec, c->stride, n, c->gc, g.elo, g.ehi, (uint8_t*)p_flag);
        if (e == cudaSuccess) e = launch_flag_count(L, (uint8_t*)p_flag, n, (int64_t*)p_chunk, (int64_t*)p_total);
        if (e == cudaSuccess) e = cudaMemcpyAsync(&g.count, p_total, sizeof(int64_t), cudaMemcpyDeviceToHost, c->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
        if (e != cudaSuccess) {
            cleanup();
            return cuda_fail(c, e, "region membership");
        }
        const int64_t stride = std::max<int64_t>((g.count + 31) / 32 * 32, 32);
        void* p = nullptr;
        if ((s = dalloc(sub, &p, (size_t)stride * R_NF * sizeof(float), "region records")) != PCT_OK) {
            s = fail(c, s, "region records: " + sub->err);
            cleanup();
            return s;
        }
        sub->d_rec = (float*)p;
        // records as the full volume computed them; the entry point's z moves
        // into the slab's grid units
        e = launch_flag_fill(L, (uint8_t*)p_flag, n, (int64_t*)p_chunk, c->d_rec, c->stride, R_NF, R_PZ,
                             (float)-g.elo, sub->d_rec, stride);
        if (e != cudaSuccess) {
            cleanup();
            return cuda_fail(c, e, "region records");
        }
        sub->n = g.count;
        sub->stride = stride;
        sub->cap = stride;
        sub->loaded = true;
        sub->rec_valid = true;
        if ((s = dalloc(sub, &p, (size_t)sg.nz * plane * sizeof(float), "region iterate")) != PCT_OK) {
            s = fail(c, s, "region iterate: " + sub->err);
            cleanup();
            return s;
        }
        g.x = (float*)p;
        e = cudaMemcpyAsync(g.x, x + (size_t)g.elo * plane, (size_t)sg.nz * plane * sizeof(float),
                            cudaMemcpyDeviceToDevice, c->stream);
        if (e != cudaSuccess) {
            cleanup();
            return cuda_fail(c, e, "region iterate copy");
        }
    }
    // 4: iterativelySolvePerGPU -- the regions one after the other on this GPU
    for (Region& g : R) {
        if (g.count == 0) continue;
        if ((s = pct_solve(g.sub, iters, lambda, block_size, g.x)) != PCT_OK) {
            s = fail(c, s, "region solve: " + g.sub->err);
            cleanup();
            return s;
        }
        c->launches += g.sub->launches;
        c->fused_launches += g.sub->fused_launches;
    }
    // 5: selectSlice -- each region's core slices make up the volume
    for (Region& g : R) {
        e = cudaMemcpyAsync(x + (size_t)g.lo * plane, g.x + (size_t)(g.lo - g.elo) * plane,
                            (size_t)(g.hi - g.lo) * plane * sizeof(float), cudaMemcpyDeviceToDevice, c->stream);
        if (e != cudaSuccess) {
            cleanup();
            return cuda_fail(c, e, "region slice copy");
        }
    }
    e = cudaStreamSynchronize(c->stream);
    unsigned flags = 0;
    for (Region& g : R) {
        unsigned f = 0;
        if (e == cudaSuccess) e = cudaMemcpy(&f, g.sub->d_flags, sizeof f, cudaMemcpyDeviceToHost);
        flags |= f;
    }
    if (region_protons)
        for (int r = 0; r < n_regions; ++r) region_protons[r] = R[(size_t)r].count;
    cleanup();
    if (e != cudaSuccess) return cuda_fail(c, e, "region solve");
    if (flags) return fail(c, PCT_ERR_DEVICE, "device check failed in a region solve (flags " + std::to_string(flags) + ")");
    return PCT_OK;
}

pct_status pct_fbp(pct_ctx* c, const pct_fbp_params* p, float* x, float* sino_out)
{
    if (!c) return PCT_ERR_ARG;
    if (!p || !x) return fail(c, PCT_ERR_ARG, "null FBP parameters or x");
    const int64_t nb = (int64_t)p->n_angle * p->n_t * p->n_v;
    if (p->n_angle < 1 || p->n_angle > fbp_max_angles() || p->n_t < 1 || p->n_t > 16384 || p->n_v < 1 ||
        nb > 0x7fffffffLL)
        return fail(c, PCT_ERR_ARG, "FBP bins: 1..4096 angles, 1..16384 t bins, >= 1 v bin, < 2^31 bins");
    if (!(p->angle_step > 0.0) || !(p->dt > 0.0) || !(p->dv > 0.0) || !std::isfinite(p->angle_step) ||
        !std::isfinite(p->dt) || !std::isfinite(p->dv) || !std::isfinite(p->t_min) || !std::isfinite(p->v_min))
        return fail(c, PCT_ERR_ARG, "FBP bin widths must be finite and > 0");
    DeviceGuard dg(c->device);
    pct_status s = need_histories(c);
    if (s != PCT_OK) return s;
    const ProtonBins P{p->n_angle, p->n_t, p->n_v, p->angle_step, p->t_min, p->dt, p->v_min, p->dv};
    void *p_cnt = nullptr, *p_sum = nullptr, *p_q = nullptr;
    if ((s = dalloc(c, &p_cnt, (size_t)nb * sizeof(unsigned), "FBP counts")) != PCT_OK ||
        (s = dalloc(c, &p_sum, (size_t)nb * sizeof(double), "FBP sums")) != PCT_OK ||
        (!sino_out && (s = dalloc(c, &p_q, (size_t)nb * sizeof(float), "FBP sinogram")) != PCT_OK)) {
        dfree(c, p_cnt);
        dfree(c, p_sum);
        return s;
    }
    float* q = sino_out ? sino_out : (float*)p_q;
    cudaError_t e = launch_fbp(launch_of(c), P, c->gc, c->d_mask, c->d_hist, c->stride, c->n, (unsigned*)p_cnt,
                               (double*)p_sum, q, x);
    // the scratch is freed once the kernels are done with it
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    dfree(c, p_cnt);
    dfree(c, p_sum);
    dfree(c, p_q);
    return e == cudaSuccess ? PCT_OK : cuda_fail(c, e, "FBP");
}

pct_status pct_tv(pct_ctx* c, const float* x, float eps, float* grad, double* value)
{
    if (!c) return PCT_ERR_ARG;
    if (!x || !grad || !value) return fail(c, PCT_ERR_ARG, "null x, grad or value");
    if (!(eps >= 0.f) || !std::isfinite(eps)) return fail(c, PCT_ERR_ARG, "eps must be finite and >= 0");
    DeviceGuard dg(c->device);
    cudaError_t e = launch_tv(launch_of(c), x, c->grid.nx, c->grid.ny, c->grid.nz, eps, grad, value);
    return e == cudaSuccess ? PCT_OK : cuda_fail(c, e, "TV kernel");
}

pct_status pct_adam(pct_ctx* c, float* x, const float* grad, float* m, float* v, int64_t n, float lr,
                    float beta1, float beta2, float eps, int32_t step)
{
    if (!c) return PCT_ERR_ARG;
    if (n < 0 || (n > 0 && (!x || !grad || !m || !v))) return fail(c, PCT_ERR_ARG, "null vector or n < 0");
    if (step < 1 || !(beta1 >= 0.f && beta1 < 1.f) || !(beta2 >= 0.f && beta2 < 1.f) ||
        !std::isfinite(lr) || !(eps > 0.f))
        return fail(c, PCT_ERR_ARG, "Adam: step >= 1, 0 <= beta < 1, eps > 0, finite lr");
    DeviceGuard dg(c->device);
    cudaError_t e = launch_adam(launch_of(c), x, grad, m, v, n, lr, beta1, beta2, eps, step);
    return e == cudaSuccess ? PCT_OK : cuda_fail(c, e, "Adam kernel");
}

pct_status pct_build_rows(pct_ctx* c)
{
    if (!c) return PCT_ERR_ARG;
    DeviceGuard dg(c->device);
    pct_status s = need_histories(c);
    if (s != PCT_OK) return s;
    return build_rows(c);
}

pct_status pct_solve_host(pct_ctx* c, int32_t iters, float lambda, int64_t block_size, float* x_host)
{
    if (!c) return PCT_ERR_ARG;
    if (!x_host) return fail(c, PCT_ERR_ARG, "null x");
    DeviceGuard dg(c->device);
    if (!c->d_xtmp) {
        void* p = nullptr;
        pct_status s = dalloc(c, &p, (size_t)c->n_vox * sizeof(float), "host-solve iterate");
        if (s != PCT_OK) return s;
        c->d_xtmp = (float*)p;
    }
    const size_t bytes = (size_t)c->n_vox * sizeof(float);
    cudaError_t e = cudaMemcpyAsync(c->d_xtmp, x_host, bytes, cudaMemcpyHostToDevice, c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "x upload");
    pct_status s = pct_solve(c, iters, lambda, block_size, c->d_xtmp);
    if (s != PCT_OK) return s;
    e = cudaMemcpyAsync(x_host, c->d_xtmp, bytes, cudaMemcpyDeviceToHost, c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "x download");
    return pct_synchronize(c);
}

namespace {

// Enqueue one batched solve on `stream`: clear barriers and accumulators,
// prepare every scan's records, launch the persistent kernel.
pct_status enqueue_batch(pct_ctx* c0, pct_ctx* const* ctxs, int32_t count, const std::vector<ScanDesc>& scans,
                         int cta, int lanes, int total, cudaStream_t stream, float* const* x)
{
    int64_t* launches = &c0->launches;
    const Launch L0{stream, c0->cta, launches};
    cudaError_t e = cudaMemsetAsync(c0->d_bar, 0, sizeof(unsigned) * count, stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(c0->d_abort, 0, sizeof(int) * count, stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(c0->d_bnext, 0, sizeof(unsigned long long) * count, stream);
    for (int32_t k = 0; k < count && e == cudaSuccess; ++k) {
        pct_ctx* c = ctxs[k];
        if (c->n == 0) continue;
        const Launch L{stream, c->cta, launches};
        e = launch_prepare(L, geo_of(c), c->d_hist, c->stride, c->n, c->d_rec);
        if (e == cudaSuccess) e = cudaMemsetAsync(c->d_acc, 0, (size_t)c->n_vox * sizeof(float2), stream);
    }
    (void)x;
    if (e == cudaSuccess)
        e = launch_drop_batch(L0, c0->d_scans, count, total, cta, lanes, c0->d_flags, (int)c0->spin_limit,
                              c0->test_unreachable);
    return e == cudaSuccess ? PCT_OK : cuda_fail(c0, e, "batched solve");
}

}  // namespace

pct_status pct_solve_batch(pct_ctx* const* ctxs, int32_t count, const int32_t* iters, const float* lambda,
                           const int64_t* block_size, float* const* x)
{
    if (!ctxs || count < 1 || !ctxs[0] || !iters || !lambda || !block_size || !x) return PCT_ERR_ARG;
    pct_ctx* c0 = ctxs[0];
    if (count > 4096) return fail(c0, PCT_ERR_ARG, "at most 4096 scans per batch");
    DeviceGuard dg(c0->device);
    int64_t work_total = 0;
    for (int32_t k = 0; k < count; ++k) {
        pct_ctx* c = ctxs[k];
        if (!c || !x[k]) return fail(c0, PCT_ERR_ARG, "null context or x in the batch");
        if (c->device != c0->device) return fail(c0, PCT_ERR_ARG, "batch contexts on different devices");
        if (!c->loaded) return fail(c0, PCT_ERR_STATE, "a batch context has no histories");
        if (iters[k] < 0 || block_size[k] < 1 || !std::isfinite(lambda[k]))
            return fail(c0, PCT_ERR_ARG, "batch iters < 0, block size < 1 or non-finite lambda");
        for (int32_t q = 0; q < k; ++q)
            if (ctxs[q] == c) return fail(c0, PCT_ERR_ARG, "a context appears twice in the batch");
        pct_status s = ensure_acc(c);
        if (s != PCT_OK) return fail(c0, s, "batch accumulator: " + c->err);
        work_total += c->n * (int64_t)iters[k];
    }
    // other contexts' pending work comes first
    for (int32_t k = 1; k < count; ++k)
        if (ctxs[k]->stream != c0->stream) cudaStreamSynchronize(ctxs[k]->stream);
    if (count > c0->scan_cap) {
        dfree(c0, c0->d_scans);
        dfree(c0, c0->d_bar);
        dfree(c0, c0->d_abort);
        dfree(c0, c0->d_bnext);
        c0->d_scans = nullptr;
        c0->d_bar = nullptr;
        c0->d_abort = nullptr;
        c0->d_bnext = nullptr;
        c0->scan_cap = 0;
        void* p = nullptr;
        pct_status s = dalloc(c0, &p, sizeof(ScanDesc) * count, "batch descriptors");
        if (s != PCT_OK) return s;
        c0->d_scans = (ScanDesc*)p;
        if ((s = dalloc(c0, &p, sizeof(unsigned) * count, "batch barriers")) != PCT_OK) return s;
        c0->d_bar = (unsigned*)p;
        if ((s = dalloc(c0, &p, sizeof(int) * count, "batch abort flags")) != PCT_OK) return s;
        c0->d_abort = (int*)p;
        if ((s = dalloc(c0, &p, sizeof(unsigned long long) * count, "batch work counters")) != PCT_OK) return s;
        c0->d_bnext = (unsigned long long*)p;
        c0->scan_cap = count;
    }
    if (pct_status sa = ensure_aux_stream(c0); sa != PCT_OK) return sa;
    // CTA size and lanes per proton: autotuned (fastest of 128 / 256 threads x
    // 32 / 16 lanes per proton on one iteration, on scratch copies of x), or
    // the context's options
    // what the tuned CTA size and the captured graph depend on (x pointers and
    // lambda live in the descriptors, uploaded before every launch)
    std::vector<int64_t> key;
    for (int32_t k = 0; k < count; ++k) {
        key.push_back((int64_t)(intptr_t)ctxs[k]);
        key.push_back(iters[k]);
        key.push_back(block_size[k]);
        key.push_back(ctxs[k]->n);
    }
    int cta = c0->cta, lanes = c0->lanes_opt;
    auto build_scans = [&](int cta_try, int lanes_try, int* total_out, std::vector<ScanDesc>& scans,
                           float* const* xs, const int32_t* its) -> pct_status {
        int cap = 0;
        cudaError_t e = batch_max_ctas(cta_try, lanes_try, c0->device, &cap);
        if (e != cudaSuccess) return cuda_fail(c0, e, "batch occupancy");
        if (cap < count) return fail(c0, PCT_ERR_ARG, "more scans than co-resident CTAs");
        scans.assign(count, ScanDesc{});
        int used = 0;
        int64_t work_left = 0;
        for (int32_t k = 0; k < count; ++k) work_left += ctxs[k]->n * (int64_t)its[k];
        for (int32_t k = 0; k < count; ++k) {
            pct_ctx* c = ctxs[k];
            ScanDesc& d = scans[k];
            const Geo G = geo_of(c);
            d.g = G.g;
            d.mc = G.mc;
            d.mask = c->d_mask;
            d.rec = c->d_rec;
            d.stride = c->stride;
            d.n = c->n;
            d.x = xs[k];
            d.acc = c->d_acc;
            d.n_vox = c->n_vox;
            d.iters = its[k];
            d.lambda = lambda[k];
            d.block = block_size[k];
            // CTAs in proportion to work, at least one each
            const int64_t wk = c->n * (int64_t)its[k];
            const int left = cap - used - (count - 1 - k);
            int share = work_left > 0 ? (int)((double)wk / (double)work_left * (cap - used)) : 1;
            if (share < 1) share = 1;
            if (share > left) share = left;
            work_left -= wk;
            d.cta0 = used;
            d.ncta = share;
            d.bar = c0->d_bar + k;
            d.abort = c0->d_abort + k;
            d.next = c0->d_bnext + k;
            used += share;
        }
        *total_out = used;
        return PCT_OK;
    };
    cudaStream_t bs = c0->batch_stream;
    cudaError_t e = cudaEventRecord(c0->batch_ev[0], c0->stream);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(bs, c0->batch_ev[0], 0);
    if (e != cudaSuccess) return cuda_fail(c0, e, "batch ordering");
    if (c0->autotune) {
        size_t hit = c0->tuned_keys.size();
        for (size_t q = 0; q < c0->tuned_keys.size(); ++q)
            if (c0->tuned_keys[q] == key) hit = q;
        if (hit < c0->tuned_keys.size()) {
            cta = c0->tuned_cta[hit];
            lanes = c0->tuned_lanes[hit];
        } else {
            // time each candidate on one iteration over scratch copies of x
            std::vector<float*> tmp(count, nullptr);
            pct_status s = PCT_OK;
            for (int32_t k = 0; k < count && s == PCT_OK; ++k) {
                void* p = nullptr;
                s = dalloc(c0, &p, (size_t)ctxs[k]->n_vox * sizeof(float), "autotune scratch");
                tmp[k] = (float*)p;
            }
            std::vector<int32_t> one(count, 1);
            float best = 1e30f;
            int best_cta = cta, best_lanes = lanes;
            cudaEvent_t t0 = nullptr, t1 = nullptr;
            cudaEventCreate(&t0);
            cudaEventCreate(&t1);
            for (int cand : {128, 256})
            for (int cand_lanes : {32, 16}) {
                if (s != PCT_OK) break;
                std::vector<ScanDesc> scans;
                int total = 0;
                if ((s = build_scans(cand, cand_lanes, &total, scans, tmp.data(), one.data())) != PCT_OK) break;
                for (int32_t k = 0; k < count; ++k)
                    cudaMemcpyAsync(tmp[k], x[k], (size_t)ctxs[k]->n_vox * sizeof(float),
                                    cudaMemcpyDeviceToDevice, bs);
                cudaMemcpyAsync(c0->d_scans, scans.data(), sizeof(ScanDesc) * count, cudaMemcpyHostToDevice, bs);
                cudaEventRecord(t0, bs);
                s = enqueue_batch(c0, ctxs, count, scans, cand, cand_lanes, total, bs, tmp.data());
                cudaEventRecord(t1, bs);
                cudaStreamSynchronize(bs);
                float ms = 0.f;
                cudaEventElapsedTime(&ms, t0, t1);
                if (s == PCT_OK && ms < best) {
                    best = ms;
                    best_cta = cand;
                    best_lanes = cand_lanes;
                }
            }
            cudaEventDestroy(t0);
            cudaEventDestroy(t1);
            for (float* p : tmp) dfree(c0, p);
            if (s != PCT_OK) return s;
            cta = best_cta;
            lanes = best_lanes;
            c0->tuned_keys.push_back(key);
            c0->tuned_cta.push_back(cta);
            c0->tuned_lanes.push_back(lanes);
        }
    }
    key.push_back(cta);
    key.push_back(lanes);
    std::vector<ScanDesc> scans;
    int total = 0;
    pct_status s = build_scans(cta, lanes, &total, scans, x, iters);
    if (s != PCT_OK) return s;
    c0->batch_cta = cta;
    c0->batch_ctas = total;
    c0->batch_lanes = lanes;
    // descriptors change only with the batch; upload them outside any graph
    e = cudaMemcpyAsync(c0->d_scans, scans.data(), sizeof(ScanDesc) * count, cudaMemcpyHostToDevice, bs);
    if (e == cudaSuccess) e = cudaStreamSynchronize(bs);
    if (e != cudaSuccess) return cuda_fail(c0, e, "batch descriptors");
    if (c0->graph) {
        if (!c0->graph_exec || c0->graph_key != key) {
            if (c0->graph_exec) cudaGraphExecDestroy(c0->graph_exec);
            c0->graph_exec = nullptr;
            cudaGraph_t g = nullptr;
            e = cudaStreamBeginCapture(bs, cudaStreamCaptureModeThreadLocal);
            if (e != cudaSuccess) return cuda_fail(c0, e, "graph capture");
            s = enqueue_batch(c0, ctxs, count, scans, cta, lanes, total, bs, x);
            cudaError_t e2 = cudaStreamEndCapture(bs, &g);
            if (s != PCT_OK) {
                if (g) cudaGraphDestroy(g);
                return s;
            }
            if (e2 != cudaSuccess) return cuda_fail(c0, e2, "graph capture");
            e = cudaGraphInstantiate(&c0->graph_exec, g, 0);
            cudaGraphDestroy(g);
            if (e != cudaSuccess) {
                c0->graph_exec = nullptr;
                return cuda_fail(c0, e, "graph instantiate");
            }
            c0->graph_key = key;
        }
        e = cudaGraphLaunch(c0->graph_exec, bs);
        if (e != cudaSuccess) return cuda_fail(c0, e, "graph launch");
        ++c0->graph_replays;
        c0->launches += 1 + count;
    } else {
        s = enqueue_batch(c0, ctxs, count, scans, cta, lanes, total, bs, x);
        if (s != PCT_OK) return s;
    }
    e = cudaEventRecord(c0->batch_ev[1], bs);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(c0->stream, c0->batch_ev[1], 0);
    return e == cudaSuccess ? PCT_OK : cuda_fail(c0, e, "batch ordering");
}

pct_status pct_synchronize(pct_ctx* c)
{
    if (!c) return PCT_ERR_ARG;
    DeviceGuard dg(c->device);
    cudaError_t e = cudaStreamSynchronize(c->stream);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(c, e, "stream");
    unsigned flags = 0;
    e = cudaMemcpy(&flags, c->d_flags, sizeof flags, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(c, e, "flag read");
    if (flags) {
        cudaMemset(c->d_flags, 0, sizeof(unsigned));
        if (flags & kFlagBarrierTimeout)
            return fail(c, PCT_ERR_TIMEOUT, "a batched-solve barrier wait gave up (spin limit reached)");
        std::string m = "device check failed:";
        if (flags & kFlagWalkGuard) m += " voxel walk step bound exceeded;";
        if (flags & kFlagHullGuard) m += " hull search step bound exceeded;";
        if (flags & kFlagMlpTable) m += " MLP sample beyond table;";
        if (flags & kFlagRowSlots) m += " a row too long for pct_rows (nnz reported as -1);";
        if (flags & kFlagPackStep) m += " packed rows: non-neighbouring consecutive voxels;";
        if (flags & kFlagRowBounds) m += " stored row length or voxel index out of range;";
        if (flags & kFlagChordRange) m += " packed rows: a chord beyond the fixed-point range (clamped);";
        return fail(c, PCT_ERR_DEVICE, m);
    }
    return PCT_OK;
}

pct_status pct_get_stat(pct_ctx* c, int32_t key, double* value)
{
    if (!c || !value) return PCT_ERR_ARG;
    DeviceGuard dg(c->device);
    switch (key) {
    case PCT_STAT_LAUNCHES: *value = (double)c->launches; return PCT_OK;
    case PCT_STAT_FUSED_LAUNCHES: *value = (double)c->fused_launches; return PCT_OK;
    case PCT_STAT_TIMED_LAUNCHES: *value = (double)(c->ev_used / 2); return PCT_OK;
    case PCT_STAT_FUSED_MS: {
        cudaError_t e = cudaStreamSynchronize(c->stream);
        if (e != cudaSuccess) return cuda_fail(c, e, "stream");
        double ms = 0.0;
        for (size_t k = 0; k + 1 < c->ev_used; k += 2) {
            float t = 0.f;
            if (cudaEventElapsedTime(&t, c->ev[k], c->ev[k + 1]) == cudaSuccess) ms += t;
        }
        cudaGetLastError();
        *value = ms;
        return PCT_OK;
    }
    case PCT_STAT_DEVICE_BYTES: *value = (double)c->mem_used; return PCT_OK;
    case PCT_STAT_N_PROTONS: *value = (double)c->n; return PCT_OK;
    case PCT_STAT_N_HULL_VOXELS: *value = (double)c->n_hull; return PCT_OK;
    case PCT_STAT_ROW_ENTRIES: *value = (double)c->nnz; return PCT_OK;
    case PCT_STAT_ROW_BYTES: *value = (double)row_bytes(c); return PCT_OK;
    case PCT_STAT_BATCH_CTA: *value = (double)c->batch_cta; return PCT_OK;
    case PCT_STAT_BATCH_CTAS: *value = (double)c->batch_ctas; return PCT_OK;
    case PCT_STAT_BATCH_LANES: *value = (double)c->batch_lanes; return PCT_OK;
    case PCT_STAT_GRAPH_REPLAYS: *value = (double)c->graph_replays; return PCT_OK;
    case PCT_STAT_SOLVE_GRAPH_REPLAYS: *value = (double)c->solve_replays; return PCT_OK;
    case PCT_STAT_WALK_FALLBACKS: {
        unsigned long long v = 0;
        cudaError_t e = cudaStreamSynchronize(c->stream);
        if (e == cudaSuccess) e = cudaMemcpy(&v, c->d_fallbacks, sizeof v, cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) return cuda_fail(c, e, "fallback counter");
        *value = (double)v;
        return PCT_OK;
    }
    default: return fail(c, PCT_ERR_ARG, "unknown stat key");
    }
}

pct_status pct_tan_angle(const double* t, double* out, int64_t n, void* cuda_stream)
{
    if (n < 0 || (n > 0 && (!t || !out))) return PCT_ERR_ARG;
    if (n == 0) return PCT_OK;
    int64_t launches = 0;
    const Launch L{(cudaStream_t)cuda_stream, 256, &launches};
    cudaError_t e = launch_tan_angle(L, t, out, n);
    if (e == cudaSuccess) e = cudaStreamSynchronize(L.stream);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return PCT_ERR_CUDA;
    }
    return PCT_OK;
}

pct_status pct_reset_stats(pct_ctx* c)
{
    if (!c) return PCT_ERR_ARG;
    if (c->d_fallbacks) {
        DeviceGuard dg(c->device);
        cudaMemsetAsync(c->d_fallbacks, 0, sizeof(unsigned long long), c->stream);
    }
    c->launches = 0;
    c->fused_launches = 0;
    c->ev_used = 0;
    return PCT_OK;
}

}  // extern "C"
