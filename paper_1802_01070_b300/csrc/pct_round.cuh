// pct_round.cuh -- one warp per proton, the row of A built round by round:
// in round r, lane l owns polyline segment 32 r + l + 1 (its MLP end point,
// its voxel walk), so every lane does the same work.  Each lane walks its
// segment with a fixed number of predicated DDA steps (the arithmetic of the
// walk in pct_warp.cuh, step for step), giving up to kPieces pieces (voxel,
// chord); pieces that continue across segment ends are joined by a warp
// segmented scan, and the finished runs (maximal visits of one voxel) are
// appended in path order to a per-warp run list in shared memory.  The row
// dot products, the residual and the DROP scatter then run lane-strided over
// that list, with no lane idle while another works.
//
// A proton whose segment needs more than kPieces - 1 crossings (the MLP step
// is longer than a voxel edge) or whose row has more runs than the list holds
// reports `fits = false`; the caller walks it with the lane-range walk of
// pct_warp.cuh instead.
#pragma once

#include "pct_warp.cuh"

namespace pct {

constexpr int kPieces = 5;          // pieces of one segment: up to 4 crossings
constexpr int kRoundRuns = 768;     // runs per warp kept in shared memory (6 KB)

struct RunList {
    int* j;      // voxel index, -1 outside the grid
    float* l;    // chord, mm
};

struct Piece {
    int j;       // linear voxel index, -1 outside the grid
    float l;
};

// Walk the segment A -> B (grid units) with kPieces - 1 predicated DDA steps.
// Returns the number of pieces; *more = the segment needs more steps.
__device__ __forceinline__ int segment_pieces(const GridC& g, float ax, float ay, float az, float bx, float by,
                                              float bz, Piece (&pc)[kPieces], bool* more)
{
    const float INF = __int_as_float(0x7f800000);
    const float Dx = bx - ax, Dy = by - ay, Dz = bz - az;
    const float ex = Dx * g.dx, ey = Dy * g.dy, ez = Dz * g.dz;
    const float l2 = fmaf(ex, ex, fmaf(ey, ey, ez * ez));
    const float len = l2 > 0.f ? l2 * rsqrtf(l2) : 0.f;
    int ix = start_index(ax, Dx), iy = start_index(ay, Dy), iz = start_index(az, Dz);
    const int sx = Dx > 0.f ? 1 : -1, sy = Dy > 0.f ? 1 : -1, sz = Dz > 0.f ? 1 : -1;
    const float rx = __fdividef(1.f, Dx), ry = __fdividef(1.f, Dy), rz = __fdividef(1.f, Dz);
    float tmx = Dx > 0.f ? (float)(ix + 1) - ax : (Dx < 0.f ? (float)ix - ax : INF);
    float tmy = Dy > 0.f ? (float)(iy + 1) - ay : (Dy < 0.f ? (float)iy - ay : INF);
    float tmz = Dz > 0.f ? (float)(iz + 1) - az : (Dz < 0.f ? (float)iz - az : INF);
    if (Dx != 0.f) tmx *= rx;
    if (Dy != 0.f) tmy *= ry;
    if (Dz != 0.f) tmz *= rz;
    const float tdx = fabsf(rx), tdy = fabsf(ry), tdz = fabsf(rz);
    float t = 0.f;
    int n = 0;
    bool open = true;
#pragma unroll
    for (int k = 0; k < kPieces - 1; ++k) {
        const float tn = fminf(tmx, fminf(tmy, tmz));
        const bool cross = open && tn < 1.f;
        const float tc = fmaxf(tn, t);
        const int j = in_grid(g, ix, iy, iz) ? lin(g, ix, iy, iz) : -1;
        if (cross) {
            pc[k].j = j;
            pc[k].l = (tc - t) * len;
            n = k + 1;
            if (tmx == tn) { ix += sx; tmx += tdx; }
            if (tmy == tn) { iy += sy; tmy += tdy; }
            if (tmz == tn) { iz += sz; tmz += tdz; }
            t = tc;
        }
        open = cross;
    }
    // the piece from the last crossing to the segment's end
    const float tn = fminf(tmx, fminf(tmy, tmz));
    *more = open && tn < 1.f;
    const int j = in_grid(g, ix, iy, iz) ? lin(g, ix, iy, iz) : -1;
#pragma unroll
    for (int k = 0; k < kPieces; ++k)
        if (k == n) {
            pc[k].j = j;
            pc[k].l = (1.f - t) * len;
        }
    return n + 1;
}

// The row of proton P in path order into the warp's run list: *total runs.
// Every lane of the warp calls it.  Returns false (and the list is not
// usable) when the proton does not fit this walk.
__device__ __forceinline__ bool round_runs(const Path& P, const MlpC& mc, const GridC& g, RunList list,
                                           int& total)
{
    const unsigned full = 0xffffffffu;
    const int lane = threadIdx.x & (kWarp - 1);
    // end point of the previous round's last segment (the entry point first)
    float cax = P.px, cay = P.py, caz = P.pz;
    // the run still open at the end of the previous round
    int open_j = 0;
    float open_l = 0.f;
    bool have_open = false;
    int base = 0;
    bool ok = true;
    for (int r0 = 0; r0 < P.nseg; r0 += kWarp) {
        const int sg = r0 + lane + 1;
        const bool act = sg <= P.nseg;
        float bx = 0.f, by = 0.f, bz = 0.f;
        if (act) path_point(P, mc, g, sg, bx, by, bz);
        float ax = __shfl_up_sync(full, bx, 1), ay = __shfl_up_sync(full, by, 1), az = __shfl_up_sync(full, bz, 1);
        if (lane == 0) {
            ax = cax;
            ay = cay;
            az = caz;
        }
        cax = __shfl_sync(full, bx, kWarp - 1);
        cay = __shfl_sync(full, by, kWarp - 1);
        caz = __shfl_sync(full, bz, kWarp - 1);
        Piece pc[kPieces];
        bool more = false;
        int np = 0;
        if (act) np = segment_pieces(g, ax, ay, az, bx, by, bz, pc, &more);
        if (__any_sync(full, more)) {
            ok = false;
            break;
        }
        // does this lane's first piece continue the previous segment's last?
        const int first_j = act ? pc[0].j : 0;
        int last_j = 0;
        float last_l = 0.f;
#pragma unroll
        for (int k = 0; k < kPieces; ++k)
            if (k == np - 1) {
                last_j = pc[k].j;
                last_l = pc[k].l;
            }
        int prev_j = __shfl_up_sync(full, last_j, 1);
        bool prev_act = __shfl_up_sync(full, (int)act, 1) != 0;
        if (lane == 0) {
            prev_j = open_j;
            prev_act = have_open;
        }
        const bool m = act && prev_act && first_j == prev_j;
        // segmented scan of the open chord: chain_l = v_l + p_l chain_(l-1)
        float v = act ? last_l : 0.f;
        bool p = act && np == 1 && m;
#pragma unroll
        for (int o = 1; o < kWarp; o <<= 1) {
            const float vu = __shfl_up_sync(full, v, o);
            const bool pu = __shfl_up_sync(full, (int)p, o) != 0;
            if (lane >= o) {
                v = p ? v + vu : v;   // (v_l, p_l) then (v_r, p_r): v_r + p_r v_l
                p = p && pu;
            }
        }
        // a chain that reaches back to lane 0 through joined lanes takes the
        // open run of the previous round
        const float chain = p ? v + (have_open ? open_l : 0.f) : v;
        float carry = __shfl_up_sync(full, chain, 1);
        if (lane == 0) carry = have_open ? open_l : 0.f;
        // the next lane continues this lane's last piece (lane 31: always,
        // into the next round; resolved there)
        const bool next_m = __shfl_down_sync(full, (int)m, 1) != 0;
        const bool cont = act && (lane == kWarp - 1 ? sg < P.nseg : next_m);
        // runs this lane completes: the previous round's open run (lane 0,
        // when not continued), then its pieces but the continued last one
        const bool emit_open = lane == 0 && have_open && !m && open_l > 0.f;
        int cnt = emit_open ? 1 : 0;
#pragma unroll
        for (int k = 0; k < kPieces; ++k) {
            if (k < np && !(k == np - 1 && cont)) {
                const float l = k == 0 && m ? pc[k].l + carry : pc[k].l;
                cnt += l > 0.f ? 1 : 0;
            }
        }
        int off = cnt;
#pragma unroll
        for (int o = 1; o < kWarp; o <<= 1) {
            const int u = __shfl_up_sync(full, off, o);
            if (lane >= o) off += u;
        }
        const int round_total = __shfl_sync(full, off, kWarp - 1);
        off = base + off - cnt;
        if (base + round_total > kRoundRuns) {
            ok = false;
            break;
        }
        if (emit_open) {
            list.j[off] = open_j;
            list.l[off] = open_l;
            ++off;
        }
#pragma unroll
        for (int k = 0; k < kPieces; ++k) {
            if (k < np && !(k == np - 1 && cont)) {
                const float l = k == 0 && m ? pc[k].l + carry : pc[k].l;
                if (l > 0.f) {
                    list.j[off] = pc[k].j;
                    list.l[off] = l;
                    ++off;
                }
            }
        }
        base += round_total;
        // the run left open by lane 31 (its chain) moves to the next round
        const float chain31 = __shfl_sync(full, chain, kWarp - 1);
        const int last31 = __shfl_sync(full, last_j, kWarp - 1);
        const bool cont31 = __shfl_sync(full, (int)cont, kWarp - 1) != 0;
        have_open = cont31;
        open_j = last31;
        open_l = chain31;
    }
    total = base;
    __syncwarp();
    return __all_sync(full, ok);
}

}  // namespace pct
