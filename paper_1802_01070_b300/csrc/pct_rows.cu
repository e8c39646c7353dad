// pct_rows.cu -- stored forms of A (built once, then streamed each iteration):
//   CSR:    int64 row offsets, int32 voxel index and FP32 chord per entry (8 B);
//   packed: int64 row offsets, the first run's voxel per row, and per entry a
//           one-byte code (3D step to the entry's voxel from the previous one,
//           plus an in-hull bit) and a 16-bit chord, fixed point or FP16 (3 B).
// Both are built by the warp walk of the fused path, so their rows are the
// fused rows; the packed form keeps the runs outside the hull too, so that
// consecutive entries are always neighbouring voxels.
#include "pct_internal.h"
#include "pct_warp.cuh"

#include <cuda_fp16.h>

namespace pct {

namespace {

constexpr int kRowCta = 256;
constexpr int kRunSlotsRows = 24;
constexpr int kScanCta = 1024;
constexpr int kScanPer = 8;                      // elements per thread
constexpr int kScanChunk = kScanCta * kScanPer;  // elements per CTA
// Step code of a packed entry: bits 0-1, 2-3 and 4-5 hold the step + 1
// (0, 1 or 2) along x, y and z; bit 6 is set when the entry's voxel is in the
// hull.
constexpr uint8_t kCodeStart = 1 | (1 << 2) | (1 << 4);   // step (0, 0, 0): the row's first run
constexpr uint8_t kCodeInside = 64;                       // bit: the entry's voxel is in the hull
constexpr int64_t kMaxRowEntries = 1 << 16;      // longer stored rows are reported, not read
// Packed rows start on groups of 4 entries (padded at their end), so that a
// lane of the DROP step loads the codes and chords of 4 entries at once.
constexpr int kPackAlign = 4;

__device__ __forceinline__ RunSlots row_slots(unsigned char* smem)
{
    const int warp = threadIdx.x >> 5;
    return RunSlots{(int2*)(smem + (size_t)warp * kRunSlotsRows * kWarp * 8)};
}

__device__ __forceinline__ int warp_sum_int(int v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ int warp_excl_scan(int v, int& total)
{
    const int lane = threadIdx.x & 31;
    int inc = v;
#pragma unroll
    for (int o = 1; o < kWarp; o <<= 1) {
        const int u = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += u;
    }
    total = __shfl_sync(0xffffffffu, inc, kWarp - 1);
    return inc - v;
}

// ---------------------------------------------------------------------------
// CSR build
// ---------------------------------------------------------------------------

__global__ void __launch_bounds__(kRowCta)
k_csr_count(GridC g, MlpC mc, RecView rv, const uint8_t* __restrict__ mask, unsigned* flags,
            int64_t m, int32_t* __restrict__ cnt)
{
    const int64_t i = blockIdx.x * (int64_t)(blockDim.x >> 5) + (threadIdx.x >> 5);
    if (i >= m) return;
    Path P;
    if (!load_path(rv, i, mc, P)) {
        if ((threadIdx.x & 31) == 0) cnt[i] = 0;
        return;
    }
    LaneWalk w;
    float s, q;
    warp_walk<0, false>(P, mc, g, mask, nullptr, flags, RunSlots{nullptr}, mc.cmin, w, s, q);
    const int mine = (w.k0 < w.k1) ? w.n - ((w.merged_prev && w.head_in) ? 1 : 0) : 0;
    const int total = warp_sum_int(mine);
    if ((threadIdx.x & 31) == 0) cnt[i] = total;
}

__global__ void __launch_bounds__(kRowCta)
k_csr_fill(GridC g, MlpC mc, RecView rv, const uint8_t* __restrict__ mask, unsigned* flags,
           int64_t m, const int64_t* __restrict__ rowptr, int32_t* __restrict__ idx,
           float* __restrict__ len)
{
    extern __shared__ unsigned char smem[];
    const int64_t i = blockIdx.x * (int64_t)(blockDim.x >> 5) + (threadIdx.x >> 5);
    if (i >= m) return;
    Path P;
    if (!load_path(rv, i, mc, P)) return;
    const RunSlots slots = row_slots(smem);
    LaneWalk w;
    float s, q;
    warp_walk<kRunSlotsRows, false>(P, mc, g, mask, nullptr, flags, slots, mc.cmin, w, s, q);
    const int mine = (w.k0 < w.k1) ? w.n - ((w.merged_prev && w.head_in) ? 1 : 0) : 0;
    int total;
    int64_t off = rowptr[i] + warp_excl_scan(mine, total);
    const int64_t end = rowptr[i + 1];
    replay_runs<kRunSlotsRows>(P, mc, g, mask, flags, slots, w, [&](int j, float l) {
        if (off < end) {
            idx[off] = j;
            len[off] = l;
        }
        ++off;
    });
}

// ---------------------------------------------------------------------------
// Packed build: every raw run (hull or not), voxels as coordinates
// ---------------------------------------------------------------------------

struct RawInfo {
    int n;                 // raw runs of the lane
    int hx, hy, hz;        // first run's voxel
    int tx, ty, tz;        // last run's voxel
    float hl, tl;
};

struct RawCount {
    RawInfo* r;
    __device__ __forceinline__ void operator()(int ix, int iy, int iz, float l)
    {
        if (r->n == 0) {
            r->hx = ix;
            r->hy = iy;
            r->hz = iz;
            r->hl = l;
        }
        r->tx = ix;
        r->ty = iy;
        r->tz = iz;
        r->tl = l;
        ++r->n;
    }
};

struct PackMerge {
    bool merged_prev, next_merges;
    float next_hl;
    int px, py, pz;        // previous lane's last voxel
};

__device__ __forceinline__ void raw_walk(const Path& P, const MlpC& mc, const GridC& g,
                                         unsigned* flags, int& k0, int& k1, RangeEnds& ends,
                                         RawInfo& r, PackMerge& pm)
{
    const int lane = threadIdx.x & 31;
    lane_range(P, mc.cmin, lane, k0, k1);
    ends = range_ends(P, mc, g, k0, k1);
    r.n = 0;
    r.hx = r.hy = r.hz = r.tx = r.ty = r.tz = 0;
    r.hl = r.tl = 0.f;
    if (k0 < k1) {
        RawCount sink{&r};
        walk_points(P, mc, g, flags, k0, k1, ends, sink);
    }
    const unsigned full = 0xffffffffu;
    pm.px = __shfl_up_sync(full, r.tx, 1);
    pm.py = __shfl_up_sync(full, r.ty, 1);
    pm.pz = __shfl_up_sync(full, r.tz, 1);
    const int pn = __shfl_up_sync(full, r.n, 1);
    pm.merged_prev = lane > 0 && pn > 0 && r.n > 0 && pm.px == r.hx && pm.py == r.hy && pm.pz == r.hz;
    // every lane takes part in each shuffle (full mask); only then the lane test
    const int nm = __shfl_down_sync(full, (int)pm.merged_prev, 1);
    pm.next_hl = __shfl_down_sync(full, r.hl, 1);
    pm.next_merges = nm != 0 && lane < kWarp - 1;
}

__global__ void __launch_bounds__(kRowCta)
k_pack_count(GridC g, MlpC mc, RecView rv, unsigned* flags, int64_t m, int32_t* __restrict__ cnt,
             short4* __restrict__ start)
{
    const int64_t i = blockIdx.x * (int64_t)(blockDim.x >> 5) + (threadIdx.x >> 5);
    if (i >= m) return;
    Path P;
    if (!load_path(rv, i, mc, P)) {
        if ((threadIdx.x & 31) == 0) {
            cnt[i] = 0;
            start[i] = make_short4(0, 0, 0, 0);
        }
        return;
    }
    int k0, k1;
    RangeEnds ends;
    RawInfo r;
    PackMerge pm;
    raw_walk(P, mc, g, flags, k0, k1, ends, r, pm);
    const int mine = r.n - (pm.merged_prev ? 1 : 0);
    const int total = warp_sum_int(mine);
    if ((threadIdx.x & 31) == 0) {
        cnt[i] = (total + kPackAlign - 1) & ~(kPackAlign - 1);   // padded to whole groups
        start[i] = make_short4((short)r.hx, (short)r.hy, (short)r.hz, 0);
    }
}

struct PackWriter {
    Dims g;
    const uint8_t* __restrict__ mask;
    unsigned* flags;
    uint8_t* codes;
    uint16_t* lens;
    float unit_inv;        // 16-bit fixed-point chords in units of 1/unit_inv mm; 0: FP16
    int64_t off, end;
    int px, py, pz;        // voxel of the previous written entry
    bool have_prev;        // px.. valid (false only for the row's very first run)
    bool skip_first;       // the first run continues the previous lane's last run
    float add_last;        // the next lane's first piece, added to the last run
    // pending run
    int qx, qy, qz;
    float ql;
    bool pending, first;
    __device__ __forceinline__ void emit(bool last)
    {
        if (!pending) return;
        if (first && skip_first) return;
        float l = ql;
        if (last) l += add_last;
        uint8_t code = kCodeStart;
        if (have_prev) {
            const int dx = qx - px, dy = qy - py, dz = qz - pz;
            if (dx < -1 || dx > 1 || dy < -1 || dy > 1 || dz < -1 || dz > 1)
                atomicOr(flags, kFlagPackStep);   // not a neighbouring voxel: cannot be coded
            else
                code = (uint8_t)((dx + 1) | ((dy + 1) << 2) | ((dz + 1) << 4));
        }
        if (g.inside(qx, qy, qz) && __ldg(mask + g.index(qx, qy, qz))) code |= kCodeInside;
        uint16_t u;
        if (unit_inv > 0.f) {
            float v = l * unit_inv;
            if (v > 65535.f) {
                atomicOr(flags, kFlagChordRange);
                v = 65535.f;
            }
            u = (uint16_t)__float2uint_rn(v);
        } else {
            u = __half_as_ushort(__float2half_rn(l));
        }
        if (off < end) {
            codes[off] = code;
            lens[off] = u;
        }
        ++off;
        px = qx;
        py = qy;
        pz = qz;
        have_prev = true;
    }
    __device__ __forceinline__ void operator()(int ix, int iy, int iz, float l)
    {
        if (pending) {
            emit(false);
            first = false;
        }
        qx = ix;
        qy = iy;
        qz = iz;
        ql = l;
        pending = true;
    }
};

__global__ void __launch_bounds__(kRowCta)
k_pack_fill(GridC g, MlpC mc, RecView rv, const uint8_t* __restrict__ mask, unsigned* flags,
            int64_t m, const int64_t* __restrict__ rowptr, uint8_t* __restrict__ codes,
            uint16_t* __restrict__ lens, float unit_inv)
{
    const int64_t i = blockIdx.x * (int64_t)(blockDim.x >> 5) + (threadIdx.x >> 5);
    if (i >= m) return;
    Path P;
    if (!load_path(rv, i, mc, P)) return;
    const int lane = threadIdx.x & 31;
    int k0, k1;
    RangeEnds ends;
    RawInfo r;
    PackMerge pm;
    raw_walk(P, mc, g, flags, k0, k1, ends, r, pm);
    const int mine = r.n - (pm.merged_prev ? 1 : 0);
    int total;
    const int64_t off = rowptr[i] + warp_excl_scan(mine, total);
    // padding entries up to the next whole group: no step, outside the hull,
    // zero chord (the decoder skips them)
    {
        const int64_t pad = rowptr[i] + total + lane;
        if (lane < kPackAlign - 1 && pad < rowptr[i + 1]) {
            codes[pad] = kCodeStart;
            lens[pad] = 0;
        }
    }
    if (k0 >= k1) return;
    // a lane other than the first codes its first run as a step from the previous
    // lane's last voxel; the row's first run is the "start" entry
    PackWriter w{Dims{g.nx, g.ny, g.nz}, mask, flags, codes, lens, unit_inv, off, rowptr[i + 1], pm.px, pm.py,
                 pm.pz, lane > 0, pm.merged_prev, pm.next_merges ? pm.next_hl : 0.f, 0, 0, 0, 0.f,
                 false, true};
    walk_points(P, mc, g, flags, k0, k1, ends, w);
    w.emit(true);
}

// ---------------------------------------------------------------------------
// Row offsets: rowptr[0] = 0, rowptr[i + 1] = cnt[0] + ... + cnt[i] (int64)
// ---------------------------------------------------------------------------

__global__ void __launch_bounds__(kScanCta)
k_scan_local(const int32_t* __restrict__ cnt, int64_t m, int64_t* __restrict__ rowptr,
             int64_t* __restrict__ chunk_sum)
{
    __shared__ int64_t warp_tot[kScanCta / 32];
    const int64_t base = blockIdx.x * (int64_t)kScanChunk + threadIdx.x * (int64_t)kScanPer;
    int64_t v[kScanPer];
    int64_t t = 0;
#pragma unroll
    for (int k = 0; k < kScanPer; ++k) {
        const int64_t e = base + k;
        t += e < m ? (int64_t)cnt[e] : 0;
        v[k] = t;
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int64_t inc = t;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int64_t u = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += u;
    }
    if (lane == 31) warp_tot[warp] = inc;
    __syncthreads();
    if (warp == 0) {
        int64_t wv = warp_tot[lane];
        int64_t wi = wv;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int64_t u = __shfl_up_sync(0xffffffffu, wi, o);
            if (lane >= o) wi += u;
        }
        warp_tot[lane] = wi - wv;
        if (lane == 31) chunk_sum[blockIdx.x] = wi;
    }
    __syncthreads();
    const int64_t before = warp_tot[warp] + inc - t;
#pragma unroll
    for (int k = 0; k < kScanPer; ++k) {
        const int64_t e = base + k;
        if (e < m) rowptr[e + 1] = before + v[k];
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) rowptr[0] = 0;
}

// Exclusive scan of the chunk sums in one CTA (sequential per thread, then warps).
__global__ void __launch_bounds__(kScanCta)
k_scan_chunks(int64_t* __restrict__ chunk_sum, int64_t nchunk)
{
    __shared__ int64_t part[kScanCta];
    const int64_t per = (nchunk + kScanCta - 1) / kScanCta;
    const int64_t a = threadIdx.x * per;
    int64_t t = 0;
    for (int64_t e = a; e < a + per && e < nchunk; ++e) t += chunk_sum[e];
    part[threadIdx.x] = t;
    __syncthreads();
    if (threadIdx.x == 0) {
        int64_t run = 0;
        for (int k = 0; k < kScanCta; ++k) {
            const int64_t u = part[k];
            part[k] = run;
            run += u;
        }
    }
    __syncthreads();
    int64_t run = part[threadIdx.x];
    for (int64_t e = a; e < a + per && e < nchunk; ++e) {
        const int64_t u = chunk_sum[e];
        chunk_sum[e] = run;
        run += u;
    }
}

__global__ void k_scan_add(int64_t* __restrict__ rowptr, int64_t m,
                           const int64_t* __restrict__ chunk_off)
{
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= m) return;
    rowptr[e + 1] += chunk_off[e / kScanChunk];
}

// ---------------------------------------------------------------------------
// DROP block step on stored rows (one warp per row)
// ---------------------------------------------------------------------------

__global__ void __launch_bounds__(kRowCta)
k_drop_csr(unsigned* flags, const int64_t* __restrict__ rowptr, const int32_t* __restrict__ idx,
           const float* __restrict__ len, const float* __restrict__ b, int64_t first,
           int64_t count, const float* __restrict__ x, float2* acc)
{
    const int64_t t = blockIdx.x * (int64_t)(blockDim.x >> 5) + (threadIdx.x >> 5);
    if (t >= count) return;
    const int64_t i = first + t;
    const int64_t a = rowptr[i], e1 = rowptr[i + 1];
    if (a == e1) return;
    if (e1 < a || e1 - a > kMaxRowEntries) {
        if ((threadIdx.x & 31) == 0) atomicOr(flags, kFlagRowBounds);
        return;
    }
    const int lane = threadIdx.x & 31;
    float s = 0.f, q = 0.f;
    // four entries per lane in flight at a time (the loop is latency-bound);
    // each lane still sums its entries in increasing order
    int64_t e = a + lane;
    for (; e + 3 * kWarp < e1; e += 4 * kWarp) {
        int j[4];
        float l[4], xv[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            j[u] = __ldg(idx + e + u * kWarp);
            l[u] = __ldg(len + e + u * kWarp);
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) xv[u] = __ldg(x + j[u]);
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            s = fmaf(l[u], xv[u], s);
            q = fmaf(l[u], l[u], q);
        }
    }
    for (; e < e1; e += kWarp) {
        const float l = __ldg(len + e);
        s = fmaf(l, __ldg(x + __ldg(idx + e)), s);
        q = fmaf(l, l, q);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        s += __shfl_xor_sync(0xffffffffu, s, o);
        q += __shfl_xor_sync(0xffffffffu, q, o);
    }
    if (!(q > 0.f)) return;
    const float r = (__ldg(b + i) - s) / q;
    e = a + lane;
    for (; e + 3 * kWarp < e1; e += 4 * kWarp) {
        int j[4];
        float l[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            j[u] = __ldg(idx + e + u * kWarp);
            l[u] = __ldg(len + e + u * kWarp);
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) atomicAdd(acc + j[u], make_float2(l[u] * r, 1.f));
    }
    for (; e < e1; e += kWarp)
        atomicAdd(acc + __ldg(idx + e), make_float2(__ldg(len + e) * r, 1.f));
}

// The codes and chords of a lane's kPackAlign entries as one load each.
template <int V>
struct PackVec;
template <>
struct PackVec<4> {
    using Codes = uint32_t;
    using Lens = uint2;
    static __device__ __forceinline__ int code(Codes c, int u) { return (int)((c >> (8 * u)) & 0xffu); }
    static __device__ __forceinline__ uint16_t len(Lens r, int u)
    {
        const uint32_t w = u < 2 ? r.x : r.y;
        return (uint16_t)((u & 1) ? (w >> 16) : (w & 0xffffu));
    }
    static __device__ __forceinline__ Codes start() { return 0x01010101u * kCodeStart; }
    static __device__ __forceinline__ Lens zero() { return make_uint2(0u, 0u); }
};

// Decode the 32 * kPackAlign entries of a packed row starting at e0 (a whole
// group): lane l takes entries e0 + kPackAlign * l .. + kPackAlign - 1 with one
// load of their codes and one of their chords, sums their steps in the lane,
// and one warp scan of the lanes' sums places them.  (bx, by, bz) is the voxel
// before e0 and is advanced past the group.  Entries at or beyond e1 decode as
// outside the hull.
__device__ __forceinline__ void unpack_group(const uint8_t* __restrict__ codes,
                                             const uint16_t* __restrict__ lens, float unit, int64_t e0,
                                             int64_t e1, int& bx, int& by, int& bz, const Dims& g,
                                             int (&j)[kPackAlign], float (&l)[kPackAlign],
                                             bool (&inside)[kPackAlign])
{
    using PV = PackVec<kPackAlign>;
    const int lane = threadIdx.x & 31;
    const int64_t e = e0 + kPackAlign * lane;
    const bool valid = e < e1;   // e1 is a whole group: all entries of the lane or none
    const typename PV::Codes cv = valid ? __ldg((const typename PV::Codes*)(codes + e)) : PV::start();
    const typename PV::Lens rv = valid ? __ldg((const typename PV::Lens*)(lens + e)) : PV::zero();
    int code[kPackAlign], p[kPackAlign];
#pragma unroll
    for (int u = 0; u < kPackAlign; ++u) {
        code[u] = PV::code(cv, u);
        // the three steps + 1 (each 0..2) into 10-bit fields
        p[u] = (code[u] & 3) | ((code[u] & 12) << 8) | ((code[u] & 48) << 16);
        if (u > 0) p[u] += p[u - 1];
    }
    int sc = p[kPackAlign - 1];
#pragma unroll
    for (int o = 1; o < kWarp; o <<= 1) {
        const int v = __shfl_up_sync(0xffffffffu, sc, o);
        if (lane >= o) sc += v;
    }
    const int excl = sc - p[kPackAlign - 1];
    const int pt = __shfl_sync(0xffffffffu, sc, 31);
#pragma unroll
    for (int u = 0; u < kPackAlign; ++u) {
        const int q = excl + p[u];
        const int c = kPackAlign * lane + u + 1;
        const int ix = bx + (q & 1023) - c, iy = by + ((q >> 10) & 1023) - c, iz = bz + ((q >> 20) & 1023) - c;
        inside[u] = valid && (code[u] & kCodeInside);
        j[u] = inside[u] ? g.index(ix, iy, iz) : 0;
        const uint16_t raw = PV::len(rv, u);
        l[u] = unit > 0.f ? (float)raw * unit : __half2float(__ushort_as_half(raw));
    }
    constexpr int kGroup = kPackAlign * kWarp;
    bx += (pt & 1023) - kGroup;
    by += ((pt >> 10) & 1023) - kGroup;
    bz += ((pt >> 20) & 1023) - kGroup;
}

// Groups of 32 * kPackAlign entries of a packed row that the DROP step decodes once and
// keeps in registers for the scatter (a torso row has ~224 entries); the
// entries beyond them are decoded again for the scatter.
constexpr int kPackedKeep = 8 / kPackAlign;

// 5 CTAs of 256 per SM (48 registers, a small spill): the step waits on its x
// gathers, and 40 resident warps measured 4 % faster than 32 at 62 registers
__global__ void __launch_bounds__(kRowCta, 5)
k_drop_packed(GridC gc, unsigned* flags, const int64_t* __restrict__ rowptr, const short4* __restrict__ start,
              const uint8_t* __restrict__ codes, const uint16_t* __restrict__ lens, float unit,
              const float* __restrict__ b, int64_t first, int64_t count,
              const float* __restrict__ x, float2* acc)
{
    const int64_t t = blockIdx.x * (int64_t)(blockDim.x >> 5) + (threadIdx.x >> 5);
    if (t >= count) return;
    const int64_t i = first + t;
    const int64_t a = rowptr[i], e1 = rowptr[i + 1];
    if (a == e1) return;
    if (e1 < a || e1 - a > kMaxRowEntries || ((a | e1) & (kPackAlign - 1))) {
        if ((threadIdx.x & 31) == 0) atomicOr(flags, kFlagRowBounds);
        return;
    }
    const Dims g{gc.nx, gc.ny, gc.nz};
    const int nvox = gc.nx * gc.ny * gc.nz;
    const short4 s0 = start[i];
    const int64_t ngroup = (e1 - a + kPackAlign * kWarp - 1) / (kPackAlign * kWarp);
    int bx = s0.x, by = s0.y, bz = s0.z;
    // the kept groups: decode all, then gather x, then accumulate in entry order
    int jk[kPackedKeep][kPackAlign];
    float lk[kPackedKeep][kPackAlign], xk[kPackedKeep][kPackAlign];
#pragma unroll
    for (int c = 0; c < kPackedKeep; ++c) {
#pragma unroll
        for (int u = 0; u < kPackAlign; ++u) {
            jk[c][u] = -1;
            lk[c][u] = 0.f;
        }
        if (c < ngroup) {   // warp-uniform
            int j[kPackAlign];
            float l[kPackAlign];
            bool in[kPackAlign];
            unpack_group(codes, lens, unit, a + c * kPackAlign * kWarp, e1, bx, by, bz, g, j, l, in);
#pragma unroll
            for (int u = 0; u < kPackAlign; ++u) {
                if (in[u] && (unsigned)j[u] >= (unsigned)nvox) {
                    atomicOr(flags, kFlagRowBounds);
                    in[u] = false;
                }
                if (in[u]) {
                    jk[c][u] = j[u];
                    lk[c][u] = l[u];
                }
            }
        }
    }
#pragma unroll
    for (int c = 0; c < kPackedKeep; ++c)
#pragma unroll
        for (int u = 0; u < kPackAlign; ++u) xk[c][u] = jk[c][u] >= 0 ? __ldg(x + jk[c][u]) : 0.f;
    float s = 0.f, q = 0.f;
#pragma unroll
    for (int c = 0; c < kPackedKeep; ++c)
#pragma unroll
        for (int u = 0; u < kPackAlign; ++u) {
            if (jk[c][u] >= 0) {
                s = fmaf(lk[c][u], xk[c][u], s);
                q = fmaf(lk[c][u], lk[c][u], q);
            }
        }
    // the rest of a long row
    const int kx = bx, ky = by, kz = bz;
    for (int64_t e0 = a + kPackedKeep * kPackAlign * kWarp; e0 < e1; e0 += kPackAlign * kWarp) {
        int j[kPackAlign];
        float l[kPackAlign];
        bool in[kPackAlign];
        unpack_group(codes, lens, unit, e0, e1, bx, by, bz, g, j, l, in);
#pragma unroll
        for (int u = 0; u < kPackAlign; ++u) {
            if (in[u] && (unsigned)j[u] >= (unsigned)nvox) {
                atomicOr(flags, kFlagRowBounds);
                in[u] = false;
            }
            if (in[u]) {
                s = fmaf(l[u], __ldg(x + j[u]), s);
                q = fmaf(l[u], l[u], q);
            }
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        s += __shfl_xor_sync(0xffffffffu, s, o);
        q += __shfl_xor_sync(0xffffffffu, q, o);
    }
    if (!(q > 0.f)) return;
    const float r = (__ldg(b + i) - s) / q;
#pragma unroll
    for (int c = 0; c < kPackedKeep; ++c)
#pragma unroll
        for (int u = 0; u < kPackAlign; ++u)
            if (jk[c][u] >= 0) atomicAdd(acc + jk[c][u], make_float2(lk[c][u] * r, 1.f));
    bx = kx;
    by = ky;
    bz = kz;
    for (int64_t e0 = a + kPackedKeep * kPackAlign * kWarp; e0 < e1; e0 += kPackAlign * kWarp) {
        int j[kPackAlign];
        float l[kPackAlign];
        bool in[kPackAlign];
        unpack_group(codes, lens, unit, e0, e1, bx, by, bz, g, j, l, in);
#pragma unroll
        for (int u = 0; u < kPackAlign; ++u)
            if (in[u] && (unsigned)j[u] < (unsigned)nvox) atomicAdd(acc + j[u], make_float2(l[u] * r, 1.f));
    }
}

inline unsigned rows_grid(int64_t n)
{
    const int wpc = kRowCta / kWarp;
    return (unsigned)((n + wpc - 1) / wpc);
}

}  // namespace

#define PCT_ROWS_TAIL(L) \
    do {                 \
        ++*(L).launches; \
        return cudaGetLastError(); \
    } while (0)

cudaError_t launch_csr_count(const Launch& L, const Geo& G, const float* rec, int64_t stride,
                             int64_t m, int32_t* cnt)
{
    if (m <= 0) return cudaSuccess;
    k_csr_count<<<rows_grid(m), kRowCta, 0, L.stream>>>(G.g, G.mc, RecView{rec, stride}, G.mask,
                                                        G.flags, m, cnt);
    PCT_ROWS_TAIL(L);
}

cudaError_t launch_csr_fill(const Launch& L, const Geo& G, const float* rec, int64_t stride,
                            int64_t m, const int64_t* rowptr, int32_t* idx, float* len)
{
    if (m <= 0) return cudaSuccess;
    const size_t sm = (size_t)(kRowCta / kWarp) * kRunSlotsRows * kWarp * 8;
    k_csr_fill<<<rows_grid(m), kRowCta, sm, L.stream>>>(G.g, G.mc, RecView{rec, stride}, G.mask,
                                                        G.flags, m, rowptr, idx, len);
    PCT_ROWS_TAIL(L);
}

cudaError_t launch_pack_count(const Launch& L, const Geo& G, const float* rec, int64_t stride,
                              int64_t m, int32_t* cnt, short4* start)
{
    if (m <= 0) return cudaSuccess;
    k_pack_count<<<rows_grid(m), kRowCta, 0, L.stream>>>(G.g, G.mc, RecView{rec, stride}, G.flags,
                                                         m, cnt, start);
    PCT_ROWS_TAIL(L);
}

cudaError_t launch_pack_fill(const Launch& L, const Geo& G, const float* rec, int64_t stride,
                             int64_t m, const int64_t* rowptr, uint8_t* codes, uint16_t* lens,
                             float chord_unit)
{
    if (m <= 0) return cudaSuccess;
    const float unit_inv = chord_unit > 0.f ? 1.f / chord_unit : 0.f;
    k_pack_fill<<<rows_grid(m), kRowCta, 0, L.stream>>>(G.g, G.mc, RecView{rec, stride}, G.mask,
                                                        G.flags, m, rowptr, codes, lens, unit_inv);
    PCT_ROWS_TAIL(L);
}

int64_t scan_chunks(int64_t m)
{
    return (m + kScanChunk - 1) / kScanChunk;
}

cudaError_t launch_row_scan(const Launch& L, const int32_t* cnt, int64_t m, int64_t* rowptr,
                            int64_t* chunk_sum)
{
    if (m <= 0) return cudaMemsetAsync(rowptr, 0, sizeof(int64_t), L.stream);
    const int64_t nc = scan_chunks(m);
    k_scan_local<<<(unsigned)nc, kScanCta, 0, L.stream>>>(cnt, m, rowptr, chunk_sum);
    k_scan_chunks<<<1, kScanCta, 0, L.stream>>>(chunk_sum, nc);
    k_scan_add<<<(unsigned)((m + 255) / 256), 256, 0, L.stream>>>(rowptr, m, chunk_sum);
    *L.launches += 3;
    return cudaGetLastError();
}

cudaError_t launch_drop_csr(const Launch& L, unsigned* flags, const int64_t* rowptr, const int32_t* idx,
                            const float* len, const float* b, int64_t first, int64_t count,
                            const float* x, float2* acc)
{
    if (count <= 0) return cudaSuccess;
    k_drop_csr<<<rows_grid(count), kRowCta, 0, L.stream>>>(flags, rowptr, idx, len, b, first, count, x, acc);
    PCT_ROWS_TAIL(L);
}

cudaError_t launch_drop_packed(const Launch& L, const GridC& g, unsigned* flags, const int64_t* rowptr,
                               const short4* start, const uint8_t* codes, const uint16_t* lens,
                               float chord_unit, const float* b, int64_t first, int64_t count,
                               const float* x, float2* acc)
{
    if (count <= 0) return cudaSuccess;
    k_drop_packed<<<rows_grid(count), kRowCta, 0, L.stream>>>(g, flags, rowptr, start, codes, lens,
                                                              chord_unit, b, first, count, x, acc);
    PCT_ROWS_TAIL(L);
}

}  // namespace pct
