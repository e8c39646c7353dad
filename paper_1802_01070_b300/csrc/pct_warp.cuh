// pct_warp.cuh -- one warp per proton: the row of A of one proton computed by
// 32 lanes cooperating (arXiv:1802.01070 maps one proton to one thread; on
// sm_103a a proton is mapped to one warp so that the lanes run in lockstep).
//
// The proton's polyline segments 1..nseg are cut into contiguous lane ranges of
// C segments (C >= cmin, the smallest count whose depth C*du exceeds a voxel
// diagonal).  Lane l computes the MLP points l*C .. (l+1)*C -- the same number
// of samples on every lane -- and walks its range.  Because a range is longer
// than any chord of a voxel, a run of the path inside one voxel can span at most
// two neighbouring lanes (the tail of lane l-1 and the head of lane l); one
// shuffle repairs the squared norm (+2ab) and decides which lane owns such a run
// for the DROP count and scatter.
//
// Pass 1 (walk): every lane stores its hull runs as (voxel, chord) pairs in
// shared memory and accumulates s = a_i.x and q = ||a_i||^2; the hull byte and
// x of a voxel are loaded when the walk steps into it and used when the run
// there ends (EntrySink), and the lane's first and last raw runs are the runs
// in the voxels its range starts and ends in.  Later passes replay the stored
// runs instead of recomputing the MLP and the walk; a lane with more runs than
// its slots re-walks its range.
#pragma once

#include "pct_device.cuh"

namespace pct {

constexpr int kWarp = 32;

// Per-warp shared-memory slots of stored runs: r[e * 32 + lane] = (voxel,
// chord bits), one 8-byte store and load per run.
struct RunSlots {
    int2* r;
    __device__ __forceinline__ void put(int e, int lane, int j, float l) const
    {
        r[e * 32 + lane] = make_int2(j, __float_as_int(l));
    }
};


// End points of a lane range: the lane computes its first point k0 and takes
// its last point k1 from the next lane (whose first point it is), so that the
// vertex two lanes share is the same float triple on both.
struct RangeEnds {
    float ax, ay, az;   // point k0
    float ex, ey, ez;   // point k1
};

// G: lanes per proton (32, or 16 with two protons per warp); every lane of the
// warp calls this.
template <int G = kWarp>
__device__ __forceinline__ RangeEnds range_ends(const Path& P, const MlpC& mc, const GridC& g,
                                                int k0, int k1)
{
    RangeEnds r;
    path_point(P, mc, g, k0, r.ax, r.ay, r.az);   // k0 >= nseg gives the exit point
    const unsigned full = 0xffffffffu;
    r.ex = __shfl_down_sync(full, r.ax, 1, G);
    r.ey = __shfl_down_sync(full, r.ay, 1, G);
    r.ez = __shfl_down_sync(full, r.az, 1, G);
    if ((threadIdx.x & (G - 1)) == G - 1) path_point(P, mc, g, k1, r.ex, r.ey, r.ez);
    return r;
}

struct LaneWalk {
    int k0, k1;          // points k0..k1 of this lane (inactive when k0 >= k1)
    RangeEnds ends;
    int n;               // hull runs met (stored while n <= RL)
    bool any;            // at least one raw run
    int head_j, tail_j;  // first / last raw run (voxel index or -1 outside the grid)
    float head_l, tail_l;
    bool head_in, tail_in;
    float s, q;          // partial a_i.x and ||a_i||^2 of the lane's runs
    bool merged_prev;    // head continues the previous lane's tail (same voxel)
    bool next_merges;    // tail continues into the next lane's head
    float next_head_l;
};

// Sinks of the walk come in two forms.  The run form has
//   on_run(ix, iy, iz, chord)  for each maximal run of the path inside one
//                              voxel (positive chord), in path order.
// The voxel-entry form (kVoxelEntry = true) has
//   start(ix, iy, iz)          the voxel the range starts in,
//   enter(ix, iy, iz)          each voxel the walk steps into,
//   emit(chord)                a run in the voxel last started or entered ends,
//   emit_last(chord)           the range's final run,
//   zero_run()                 a run of zero length was met (nothing emitted),
// so that a sink can fetch what it needs of a voxel as soon as the walk steps
// into it, one crossing before the run there is emitted.
template <class F, class = void>
struct VoxelEntrySink {
    static constexpr bool value = false;
};
template <class F>
struct VoxelEntrySink<F, decltype((void)F::kVoxelEntry)> {
    static constexpr bool value = F::kVoxelEntry;
};

// Walk the points k0..k1 of P (ends given), reporting to the sink on_run.
template <class F>
__device__ __forceinline__ void walk_points(const Path& P, const MlpC& mc, const GridC& g,
                                            unsigned* flags, int k0, int k1, const RangeEnds& re,
                                            F& on_run)
{
    float ax = re.ax, ay = re.ay, az = re.az, bx, by, bz;
    if (k0 + 1 == k1) {
        bx = re.ex;
        by = re.ey;
        bz = re.ez;
    } else {
        path_point(P, mc, g, k0 + 1, bx, by, bz);
    }
    int ix = start_index(ax, bx - ax);
    int iy = start_index(ay, by - ay);
    int iz = start_index(az, bz - az);
    constexpr bool kEntry = VoxelEntrySink<F>::value;
    if constexpr (kEntry) on_run.start(ix, iy, iz);
    float run = 0.f;
    const float INF = __int_as_float(0x7f800000);
    for (int k = k0 + 1; k <= k1; ++k) {
        if (k > k0 + 1) {
            if (k == k1) {
                bx = re.ex;
                by = re.ey;
                bz = re.ez;
            } else {
                path_point(P, mc, g, k, bx, by, bz);
            }
        }
        const float Dx = bx - ax, Dy = by - ay, Dz = bz - az;
        const float ex = Dx * g.dx, ey = Dy * g.dy, ez = Dz * g.dz;
        const float l2 = fmaf(ex, ex, fmaf(ey, ey, ez * ez));
        const float len = l2 > 0.f ? l2 * rsqrtf(l2) : 0.f;
        const bool px = Dx > 0.f, py = Dy > 0.f, pz = Dz > 0.f;
        const int sx = px ? 1 : -1, sy = py ? 1 : -1, sz = pz ? 1 : -1;
        const float rx = __fdividef(1.f, Dx), ry = __fdividef(1.f, Dy), rz = __fdividef(1.f, Dz);
        // parameter of the first face crossed on each axis ((float)ix + 1 is
        // exact: grids hold fewer than 2^24 voxels along an axis); none on an
        // axis the segment does not move along
        float tmx = Dx != 0.f ? ((float)ix + (px ? 1.f : 0.f) - ax) * rx : INF;
        float tmy = Dy != 0.f ? ((float)iy + (py ? 1.f : 0.f) - ay) * ry : INF;
        float tmz = Dz != 0.f ? ((float)iz + (pz ? 1.f : 0.f) - az) * rz : INF;
        const float tdx = fabsf(rx), tdy = fabsf(ry), tdz = fabsf(rz);
        const int guard = (int)(fabsf(Dx) + fabsf(Dy) + fabsf(Dz)) + 4;
        float t = 0.f;
        int nstep = 0;
        for (;;) {
            const float tn = fminf(tmx, fminf(tmy, tmz));
            if (!(tn < 1.f) || nstep > guard) {
                if (nstep > guard)
                    atomicOr(flags, kFlagWalkGuard);
                else
                    run = fmaf(1.f - t, len, run);
                break;
            }
            const float tc = fmaxf(tn, t);
            run = fmaf(tc - t, len, run);
            if constexpr (kEntry) {
                if (run > 0.f)
                    on_run.emit(run);
                else
                    on_run.zero_run();
            } else {
                if (run > 0.f) on_run(ix, iy, iz, run);
            }
            run = 0.f;
            if (tmx == tn) { ix += sx; tmx += tdx; }
            if (tmy == tn) { iy += sy; tmy += tdy; }
            if (tmz == tn) { iz += sz; tmz += tdz; }
            if constexpr (kEntry) on_run.enter(ix, iy, iz);
            t = tc;
            ++nstep;
        }
        ax = bx;
        ay = by;
        az = bz;
    }
    if constexpr (kEntry) {
        if (run > 0.f)
            on_run.emit_last(run);
        else
            on_run.zero_run();
    } else {
        if (run > 0.f) on_run(ix, iy, iz, run);
    }
}

// Grid extent a sink needs (passed by value: taking the address of a kernel
// parameter would force a stack copy).
struct Dims {
    int nx, ny, nz;
    __device__ __forceinline__ bool inside(int ix, int iy, int iz) const
    {
        return (unsigned)ix < (unsigned)nx && (unsigned)iy < (unsigned)ny && (unsigned)iz < (unsigned)nz;
    }
    __device__ __forceinline__ int index(int ix, int iy, int iz) const { return ix + nx * (iy + ny * iz); }
};

// Pass-1 sink in the voxel-entry form: the hull byte (and x) of a voxel are
// loaded when the walk steps into it and used when the run there ends, one
// crossing later, so the loads overlap the walk's arithmetic with no per-run
// copies.  Hull runs are counted, accumulated into s = a_i.x and q =
// ||a_i||^2 and stored (the first RL).  With no run of zero length, the lane's
// first raw run lies in the voxel its range starts in and its last raw run in
// the voxel the range ends in; a zero-length run sets `odd`, and the caller
// then walks the lane again with StoreSink.
// CG: read x through L2 only (ld.global.cg), for kernels in which other CTAs
// rewrite x between barriers; otherwise the read-only cache path.
template <int RL, bool DOT, bool CG = false>
struct EntrySink {
    static constexpr bool kVoxelEntry = true;
    Dims g;
    const uint8_t* __restrict__ mask;
    const float* __restrict__ x;
    RunSlots slots;
    int lane;
    int n;
    float s, q;
    int j, j0;     // voxel the walk is in, voxel the range starts in (-1 outside the grid)
    float xv;      // x of voxel j (DOT)
    float last;    // chord of the range's final run
    uint8_t m;     // hull byte of voxel j
    bool odd;

    __device__ __forceinline__ void enter(int ix, int iy, int iz)
    {
        j = -1;
        m = 0;
        xv = 0.f;
        if (g.inside(ix, iy, iz)) {
            j = g.index(ix, iy, iz);
            m = __ldg(mask + j);
            if (DOT) xv = CG ? __ldcg(x + j) : __ldg(x + j);
        }
    }
    __device__ __forceinline__ void start(int ix, int iy, int iz)
    {
        enter(ix, iy, iz);
        j0 = j;
    }
    __device__ __forceinline__ void emit(float l)
    {
        if (m) {
            if (DOT) s = fmaf(l, xv, s);
            q = fmaf(l, l, q);
            if (n < RL) slots.put(n, lane, j, l);
            ++n;
        }
    }
    __device__ __forceinline__ void emit_last(float l)
    {
        emit(l);
        last = l;
    }
    __device__ __forceinline__ void zero_run() { odd = true; }
};

// Pass-1 sink in the run form (the exact fallback of EntrySink, and the walk
// of kernels without run slots): the hull byte (and x) of a run are loaded
// when the run is emitted and used when the next run is emitted.
template <int RL, bool DOT, bool CG = false>
struct StoreSink {
    Dims g;
    const uint8_t* __restrict__ mask;
    const float* __restrict__ x;
    RunSlots slots;
    int lane;
    LaneWalk* w;
    int pj;
    float pl, px;
    uint8_t pm;
    bool pending;

    // the pending run (there is one) is final: count, accumulate and store it
    __device__ __forceinline__ void commit()
    {
        if (pm) {
            if (DOT) w->s = fmaf(pl, px, w->s);
            w->q = fmaf(pl, pl, w->q);
            if (w->n < RL) slots.put(w->n, lane, pj, pl);
            ++w->n;
        }
    }
    __device__ __forceinline__ void operator()(int ix, int iy, int iz, float l)
    {
        int j = -1;
        uint8_t m = 0;
        float xv = 0.f;
        if (g.inside(ix, iy, iz)) {
            j = g.index(ix, iy, iz);
            m = __ldg(mask + j);
            if (DOT) xv = CG ? __ldcg(x + j) : __ldg(x + j);
        }
        if (pending) {
            commit();
        } else {   // the lane's first raw run
            w->head_j = j;
            w->head_l = l;
        }
        pj = j;
        pl = l;
        px = xv;
        pm = m;
        pending = true;
    }
};

// Lane range of a proton with nseg segments (lane of G).
template <int G = kWarp>
__device__ __forceinline__ void lane_range(const Path& P, int cmin, int lane, int& k0, int& k1)
{
    int C = (P.nseg + G - 1) / G;
    if (C < cmin) C = cmin;
    k0 = lane * C;
    k1 = min(k0 + C, P.nseg);
}

// Pass 1 for the proton P on the calling group of G lanes (the whole warp, or
// one half of it): walk, store, accumulate, and resolve the runs shared by
// neighbouring lanes.  Returns the group-reduced (s, q) on every lane of the
// group.  Every lane of the warp must call it (the shuffles span the warp); a
// group without a proton passes nseg = 0.  Run slots are indexed by warp lane.
template <int RL, bool DOT, bool CG = false, int G = kWarp>
__device__ __forceinline__ void warp_walk(const Path& P, const MlpC& mc, const GridC& g,
                                          const uint8_t* __restrict__ mask,
                                          const float* __restrict__ x, unsigned* flags,
                                          RunSlots slots, int cmin, LaneWalk& w, float& s_all,
                                          float& q_all)
{
    const int wl = threadIdx.x & (kWarp - 1);
    const int lane = threadIdx.x & (G - 1);
    lane_range<G>(P, cmin, lane, w.k0, w.k1);
    w.n = 0;
    w.any = false;
    w.head_j = w.tail_j = -1;
    w.head_l = w.tail_l = 0.f;
    w.head_in = w.tail_in = false;
    w.s = w.q = 0.f;
    w.ends = range_ends<G>(P, mc, g, w.k0, w.k1);
    bool exact = RL == 0;
    if (RL > 0 && w.k0 < w.k1) {
        EntrySink<RL, DOT, CG> sink{Dims{g.nx, g.ny, g.nz}, mask, x, slots, wl, 0, 0.f, 0.f, -1, -1, 0.f, 0.f, 0, false};
        walk_points(P, mc, g, flags, w.k0, w.k1, w.ends, sink);
        if (!sink.odd) {
            w.n = sink.n;
            w.s = sink.s;
            w.q = sink.q;
            w.any = true;
            w.tail_j = sink.j;
            w.tail_l = sink.last;
            w.tail_in = sink.m != 0;
            w.head_j = sink.j0;
            // the first raw run is a hull run exactly when it is the first
            // stored run (a voxel outside the hull is never stored, and a
            // later hull run lies in another voxel); only then does its
            // chord matter
            w.head_in = w.n > 0 && w.head_j >= 0 && slots.r[wl].x == w.head_j;
            if (w.head_in) w.head_l = __int_as_float(slots.r[wl].y);
        } else {
            exact = true;
        }
    }
    if (exact && w.k0 < w.k1) {
        StoreSink<RL, DOT, CG> sink{Dims{g.nx, g.ny, g.nz}, mask, x, slots, wl, &w, -1, 0.f, 0.f, 0, false};
        walk_points(P, mc, g, flags, w.k0, w.k1, w.ends, sink);
        if (sink.pending) {
            sink.commit();
            // the pending run after the walk is the lane's last raw run
            w.any = true;
            w.tail_j = sink.pj;
            w.tail_l = sink.pl;
            w.tail_in = sink.pm != 0;
            // the first raw run is a hull run exactly when it is the first
            // stored run: a voxel outside the hull is never stored, and a
            // later hull run lies in another voxel
            if (RL > 0)
                w.head_in = w.n > 0 && w.head_j >= 0 && slots.r[wl].x == w.head_j;
            else
                w.head_in = w.head_j >= 0 && __ldg(mask + w.head_j) != 0;
        }
    }
    const unsigned full = 0xffffffffu;
    const int pt_j = __shfl_up_sync(full, w.tail_j, 1, G);
    const float pt_l = __shfl_up_sync(full, w.tail_l, 1, G);
    const bool p_any = __shfl_up_sync(full, (int)w.any, 1, G) != 0;
    w.merged_prev = lane > 0 && p_any && w.any && w.head_j >= 0 && pt_j == w.head_j;
    w.next_merges = __shfl_down_sync(full, (int)w.merged_prev, 1, G) != 0 && lane < G - 1;
    w.next_head_l = __shfl_down_sync(full, w.head_l, 1, G);
    float q = w.q;
    if (w.merged_prev && w.head_in) q = fmaf(2.f * pt_l, w.head_l, q);
    float s = w.s;
#pragma unroll
    for (int o = G / 2; o > 0; o >>= 1) {
        s += __shfl_xor_sync(full, s, o, G);
        q += __shfl_xor_sync(full, q, o, G);
    }
    s_all = s;
    q_all = q;
}

// Scatter sink used when a lane re-walks its range (more runs than slots):
// drops the head run owned by the previous lane and extends the tail run by the
// next lane's head piece.
template <class Op>
struct RewalkSink {
    Dims g;
    const uint8_t* __restrict__ mask;
    const LaneWalk* w;
    Op op;
    int pj;
    float pl;
    uint8_t pm;
    bool pending, first;
    __device__ __forceinline__ void flush(bool last)
    {
        if (!pending || !pm) return;
        if (first && w->merged_prev) return;
        float l = pl;
        if (last && w->next_merges) l += w->next_head_l;
        op(pj, l);
    }
    __device__ __forceinline__ void operator()(int ix, int iy, int iz, float l)
    {
        int j = -1;
        uint8_t m = 0;
        if (g.inside(ix, iy, iz)) {
            j = g.index(ix, iy, iz);
            m = __ldg(mask + j);
        }
        if (pending) {
            flush(false);
            first = false;
        }
        pj = j;
        pl = l;
        pm = m;
        pending = true;
    }
};

// Replay (or re-walk) this lane's hull runs with their final ownership:
// op(j, chord) once per run of the row.
template <int RL, class Op>
__device__ __forceinline__ void replay_runs(const Path& P, const MlpC& mc, const GridC& g,
                                            const uint8_t* __restrict__ mask, unsigned* flags,
                                            RunSlots slots, const LaneWalk& w, Op op)
{
    if (w.k0 >= w.k1) return;
    const int lane = threadIdx.x & (kWarp - 1);
    if (w.n <= RL) {
        // the head run goes to the previous lane when it continues that
        // lane's tail; the tail run takes the next lane's head piece
        const int e0 = (w.merged_prev && w.head_in) ? 1 : 0;
        const int last = w.n - 1;
        const float ext = (w.next_merges && w.tail_in) ? w.next_head_l : 0.f;
        for (int e = e0; e < w.n; ++e) {
            const int2 v = slots.r[e * kWarp + lane];
            float l = __int_as_float(v.y);
            if (e == last) l += ext;
            op(v.x, l);
        }
    } else {
        RewalkSink<Op> sink{Dims{g.nx, g.ny, g.nz}, mask, &w, op, -1, 0.f, 0, false, true};
        walk_points(P, mc, g, flags, w.k0, w.k1, w.ends, sink);
        sink.flush(true);
    }
}

}  // namespace pct
