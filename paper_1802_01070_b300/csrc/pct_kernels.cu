// pct_kernels.cu -- CUDA kernels of libpct and their launchers (sm_103a).
//
// The record kernel maps one proton to one thread, as arXiv:1802.01070 maps
// every proton (Sec. I); the kernels that walk paths map one proton to one
// warp (pct_warp.cuh) and recompute the proton's row of A from its record:
// MLP samples, then the voxel walk.  None of them stores A.  Also here: the
// valid-proton lists of the DROP blocks and the hull distance map.
#include "pct_internal.h"
#include "pct_round.cuh"
#include "pct_warp.cuh"

namespace pct {

namespace {

constexpr int kMaxCta = 512;

inline unsigned grid_for(int64_t n, int cta)
{
    return (unsigned)((n + cta - 1) / cta);
}

// ---------------------------------------------------------------------------
// Hull-frame record of each proton: rotate the tracker data into the
// beam frame of its gantry angle, follow both straight tracker lines to the
// hull, and store the entry/exit states the MLP starts from.
// ---------------------------------------------------------------------------
// Crossing parameter (mm of depth) of the lab line p(s) = T + s D with the grid
// plane `face` of `axis`, in FP64.
__device__ __forceinline__ double plane_crossing(const GridC& g, const double T[3], const double D[3],
                                                 int axis, int face)
{
    if (axis < 0) return 0.0;
    const double o = axis == 0 ? (double)g.ox : (axis == 1 ? (double)g.oy : (double)g.oz);
    const double d = axis == 0 ? (double)g.dx : (axis == 1 ? (double)g.dy : (double)g.dz);
    return (fma((double)face, d, o) - T[axis]) / D[axis];
}

// tan t of a tracker angle.  For |t| <= 0.25 rad (nearly every proton) the
// Maclaurin series tan t = sum_n T_n t^(2n-1), T_n = (-1)^(n-1) 2^(2n)
// (2^(2n) - 1) B_2n / (2n)! with B the Bernoulli numbers, summed to 11 terms
// in Horner form in t^2 (relative error within 2.3e-16, about one unit in the
// last place, on that range, checked
// against 40-digit arithmetic); larger angles take the library tan.
__device__ __forceinline__ double tan_angle(double t)
{
    if (!(fabs(t) <= 0.25)) return tan(t);
    constexpr double T[11] = {1.0,
                              1.0 / 3.0,
                              2.0 / 15.0,
                              17.0 / 315.0,
                              62.0 / 2835.0,
                              1382.0 / 155925.0,
                              21844.0 / 6081075.0,
                              929569.0 / 638512875.0,
                              6404582.0 / 10854718875.0,
                              443861162.0 / 1856156927625.0,
                              18888466084.0 / 194896477400625.0};
    const double t2 = t * t;
    double a = T[10];
#pragma unroll
    for (int k = 9; k >= 0; --k) a = fma(a, t2, T[k]);
    return a * t;
}

__global__ void k_tan_angle(const double* __restrict__ t, double* __restrict__ out, int64_t n)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) out[i] = tan_angle(t[i]);
}

__global__ void __launch_bounds__(kMaxCta)
k_prepare(GridC g, const uint8_t* __restrict__ mask, const uint8_t* __restrict__ dist, unsigned* flags,
          const float* __restrict__ h,
          int64_t stride, int64_t first, int64_t count, float* __restrict__ rec, float Lmax)
{
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= count) return;
    const int64_t i = first + t;
    const float xi = h[H_INX * stride + i], yi = h[H_INY * stride + i], zi = h[H_INZ * stride + i];
    const float xo = h[H_OUTX * stride + i], yo = h[H_OUTY * stride + i], zo = h[H_OUTZ * stride + i];
    const float thi = h[H_THI * stride + i], psi = h[H_PSI * stride + i];
    const float tho = h[H_THO * stride + i], pso = h[H_PSO * stride + i];
    const float phi = h[H_PHI * stride + i], wepl = h[H_WEPL * stride + i];
    float s, c;
    sincosf(phi, &s, &c);
    const float ua = fmaf(xi, c, yi * s), ub = fmaf(xo, c, yo * s);
    const float tti = tanf(thi), tpi = tanf(psi), tto = tanf(tho), tpo = tanf(pso);
    bool ok = isfinite(xi) && isfinite(yi) && isfinite(zi) && isfinite(xo) && isfinite(yo) &&
              isfinite(zo) && isfinite(ua) && isfinite(ub) && isfinite(tti) && isfinite(tpi) &&
              isfinite(tto) && isfinite(tpo) && ub > ua;
    const float S = ub - ua;
    // FP32 search of the first hull voxel along each straight tracker line
    // (grid units per mm of depth)
    const float Tix = (xi - g.ox) * g.idx, Tiy = (yi - g.oy) * g.idy, Tiz = (zi - g.oz) * g.idz;
    const float Dix = fmaf(-tti, s, c) * g.idx, Diy = fmaf(tti, c, s) * g.idy, Diz = tpi * g.idz;
    const float Tox = (xo - g.ox) * g.idx, Toy = (yo - g.oy) * g.idy, Toz = (zo - g.oz) * g.idz;
    const float Dox = -fmaf(-tto, s, c) * g.idx, Doy = -fmaf(tto, c, s) * g.idy, Doz = -tpo * g.idz;
    float s_in = 0.f, s_out = 0.f;
    int ax_in = -1, f_in = 0, ax_out = -1, f_out = 0;
    if (ok) ok = hull_entry(g, mask, dist, Tix, Tiy, Tiz, Dix, Diy, Diz, S, flags, s_in, ax_in, f_in);
    if (ok) ok = hull_entry(g, mask, dist, Tox, Toy, Toz, Dox, Doy, Doz, S, flags, s_out, ax_out, f_out);
    // the record, evaluated once in FP64 from the raw inputs and the crossed planes
    double sd, cd;
    sincos((double)phi, &sd, &cd);
    const double ti = tan_angle(thi), pi = tan_angle(psi), to = tan_angle(tho), po = tan_angle(pso);
    const double Ti[3] = {xi, yi, zi}, To[3] = {xo, yo, zo};
    const double Di[3] = {fma(-ti, sd, cd), fma(ti, cd, sd), pi};
    const double Do[3] = {-fma(-to, sd, cd), -fma(to, cd, sd), -po};
    const double si = ok ? plane_crossing(g, Ti, Di, ax_in, f_in) : 0.0;
    const double so = ok ? plane_crossing(g, To, Do, ax_out, f_out) : 0.0;
    const double uad = fma((double)xi, cd, (double)yi * sd), ubd = fma((double)xo, cd, (double)yo * sd);
    const double tad = fma(-(double)xi, sd, (double)yi * cd), tbd = fma(-(double)xo, sd, (double)yo * cd);
    const double u_in = uad + si, u_out = ubd - so;
    const double L = u_out - u_in;
    ok = ok && L > 0.0 && L <= (double)Lmax;
    rec[R_C * stride + i] = (float)cd;
    rec[R_S * stride + i] = (float)sd;
    rec[R_UIN * stride + i] = (float)u_in;
    rec[R_L * stride + i] = ok ? (float)L : 0.f;
    rec[R_T0 * stride + i] = (float)fma(ti, si, tad);
    rec[R_TH0 * stride + i] = thi;
    rec[R_V0 * stride + i] = (float)fma(pi, si, (double)zi);
    rec[R_PS0 * stride + i] = psi;
    rec[R_T2 * stride + i] = (float)fma(-to, so, tbd);
    rec[R_TH2 * stride + i] = tho;
    rec[R_V2 * stride + i] = (float)fma(-po, so, (double)zo);
    rec[R_PS2 * stride + i] = pso;
    rec[R_PX * stride + i] = (float)((fma(si, Di[0], Ti[0]) - (double)g.ox) / (double)g.dx);
    rec[R_PY * stride + i] = (float)((fma(si, Di[1], Ti[1]) - (double)g.oy) / (double)g.dy);
    rec[R_PZ * stride + i] = (float)((fma(si, Di[2], Ti[2]) - (double)g.oz) / (double)g.dz);
    rec[R_B * stride + i] = wepl;
}

// Chessboard distance of every voxel to the nearest hull voxel, capped at 255
// (the skipping table of the hull search), in three separable passes:
//   f1(v) = min over hull voxels h of its x row      |v_x - h_x|
//   f2(v) = min over y' of max(|v_y - y'|, f1(v_x, y', v_z))
//   f3(v) = min over z' of max(|v_z - z'|, f2(v_x, v_y, z'))
// which is min over hull voxels h of max(|v_x-h_x|, |v_y-h_y|, |v_z-h_z|).
__global__ void k_hull_dist_x(const uint8_t* __restrict__ mask, int nx, int64_t rows,
                              uint8_t* __restrict__ out)
{
    const int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (r >= rows) return;
    const uint8_t* m = mask + r * nx;
    uint8_t* o = out + r * nx;
    int last = -1;
    for (int x = 0; x < nx; ++x) {
        if (m[x]) last = x;
        o[x] = (uint8_t)(last < 0 ? 255 : min(x - last, 255));
    }
    last = -1;
    for (int x = nx - 1; x >= 0; --x) {
        if (m[x]) last = x;
        if (last >= 0) o[x] = (uint8_t)min((int)o[x], min(last - x, 255));
    }
}

// One of the min-max passes along an axis of n voxels with element stride
// `stride` (f2 from f1 along y, f3 from f2 along z).
__global__ void k_hull_dist_axis(const uint8_t* __restrict__ in, int n, int64_t stride, int64_t n_vox,
                                 uint8_t* __restrict__ out)
{
    const int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (v >= n_vox) return;
    const int a = (int)((v / stride) % n);
    int best = in[v];
    for (int r = 1; r < best; ++r) {
        if (a - r >= 0) best = min(best, max(r, (int)in[v - r * stride]));
        if (a + r < n) best = min(best, max(r, (int)in[v + r * stride]));
    }
    out[v] = (uint8_t)best;
}

__global__ void k_hull_states(const float* __restrict__ rec, int64_t stride, int64_t first,
                              int64_t count, float* __restrict__ out)
{
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= count) return;
    const int64_t i = first + t;
    const float L = rec[R_L * stride + i];
    const float u_in = rec[R_UIN * stride + i];
    float* o = out + 12 * t;
    o[0] = u_in;
    o[1] = u_in + L;
    o[2] = rec[R_T0 * stride + i];
    o[3] = rec[R_TH0 * stride + i];
    o[4] = rec[R_V0 * stride + i];
    o[5] = rec[R_PS0 * stride + i];
    o[6] = rec[R_T2 * stride + i];
    o[7] = rec[R_TH2 * stride + i];
    o[8] = rec[R_V2 * stride + i];
    o[9] = rec[R_PS2 * stride + i];
    o[10] = L > 0.f ? 1.f : 0.f;
    o[11] = 0.f;
}

// MLP polyline in lab mm (debug / parity).
__global__ void __launch_bounds__(kMaxCta)
k_mlp_points(GridC g, MlpC mc, RecView rv, int64_t first, int64_t count, int32_t max_pts,
             float* __restrict__ out, int32_t* __restrict__ npts)
{
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= count) return;
    Path P;
    if (!load_path(rv, first + t, mc, P)) {
        npts[t] = 0;
        return;
    }
    npts[t] = P.nseg + 1;
    const int last = P.nseg < max_pts - 1 ? P.nseg : max_pts - 1;
    for (int k = 0; k <= last; ++k) {
        float x, y, z;
        path_point(P, mc, g, k, x, y, z);
        float* o = out + ((int64_t)t * max_pts + k) * 3;
        o[0] = fmaf(x, g.dx, g.ox);
        o[1] = fmaf(y, g.dy, g.oy);
        o[2] = fmaf(z, g.dz, g.oz);
    }
}

// Runs a lane can keep in shared memory: DROP / adjoint passes, and the debug
// row writer (which must not fall back).
constexpr int kRunSlots = 24;
// warp-per-proton kernels: at most 256 threads per CTA, 3 CTAs per SM (80
// registers per thread, no spills: measured faster than 4 CTAs with spills)
constexpr int kWarpCta = 256;
constexpr int kWarpCtaMin = 3;
constexpr int kRowSlots = 64;

__device__ __forceinline__ RunSlots warp_slots(unsigned char* smem, int rl)
{
    const int warp = threadIdx.x >> 5;
    return RunSlots{(int2*)(smem + (size_t)warp * rl * kWarp * 8)};
}

// The same bytes as the round walk's run list (voxel array, then chord array).
__device__ __forceinline__ RunList warp_list(unsigned char* smem, int rl)
{
    const int warp = threadIdx.x >> 5;
    unsigned char* base = smem + (size_t)warp * rl * kWarp * 8;
    return RunList{(int*)base, (float*)(base + (size_t)rl * kWarp * 4)};
}

// Rows of A in path order (debug / parity), one warp per proton.
__global__ void __launch_bounds__(kMaxCta)
k_rows(GridC g, MlpC mc, RecView rv, const uint8_t* __restrict__ mask, unsigned* flags,
       int64_t first, int64_t count, int32_t max_nnz, int32_t* __restrict__ idx,
       float* __restrict__ len, int32_t* __restrict__ nnz)
{
    extern __shared__ unsigned char smem[];
    const int lane = threadIdx.x & (kWarp - 1);
    const int64_t t = blockIdx.x * (int64_t)(blockDim.x >> 5) + (threadIdx.x >> 5);
    if (t >= count) return;
    Path P;
    if (!load_path(rv, first + t, mc, P)) {
        if (lane == 0) nnz[t] = 0;
        return;
    }
    const RunSlots slots = warp_slots(smem, kRowSlots);
    LaneWalk w;
    float s, q;
    warp_walk<kRowSlots, false>(P, mc, g, mask, nullptr, flags, slots, mc.cmin, w, s, q);
    const bool over = __any_sync(0xffffffffu, w.n > kRowSlots);
    if (over) {
        if (lane == 0) {
            nnz[t] = -1;
            atomicOr(flags, kFlagRowSlots);
        }
        return;
    }
    int mine = (w.k0 < w.k1) ? w.n - ((w.merged_prev && w.head_in) ? 1 : 0) : 0;
    int off = mine;
#pragma unroll
    for (int o = 1; o < kWarp; o <<= 1) {
        const int v = __shfl_up_sync(0xffffffffu, off, o);
        if (lane >= o) off += v;
    }
    const int total = __shfl_sync(0xffffffffu, off, kWarp - 1);
    off -= mine;
    int32_t* oi = idx + t * (int64_t)max_nnz;
    float* ol = len + t * (int64_t)max_nnz;
    replay_runs<kRowSlots>(P, mc, g, mask, flags, slots, w, [&](int j, float l) {
        if (off < max_nnz) {
            oi[off] = j;
            ol[off] = l;
        }
        ++off;
    });
    if (lane == 0) nnz[t] = total;
}

// Work distribution of the warp-per-proton kernels: the grid has one warp per
// item up to filling the GPU once.  Each warp takes a first chunk of `first`
// items by its index (kGrab when there are at least kGrab items per warp of
// the grid, else 1) and, while items are left, chunks of kGrab items from the
// counter *next (zero at launch), so that warps whose paths were short take
// more of them and the launch ends evenly.  body(t) runs on the whole warp.
constexpr int kGrab = 2;

template <class F>
__device__ __forceinline__ void for_each_item(int64_t count, int first, unsigned long long* next, F&& body)
{
    const int64_t stat = (int64_t)gridDim.x * (blockDim.x >> 5) * first;   // items assigned by index
    const int lane = threadIdx.x & (kWarp - 1);
    int64_t base = (blockIdx.x * (int64_t)(blockDim.x >> 5) + (threadIdx.x >> 5)) * first;
    int64_t end = base + first;
    while (base < count) {
        end = end < count ? end : count;
        for (int64_t t = base; t < end; ++t) body(t);
        if (stat >= count) break;   // every item was assigned by index
        unsigned long long got = 0;
        if (lane == 0) got = atomicAdd(next, (unsigned long long)kGrab);
        base = stat + (int64_t)__shfl_sync(0xffffffffu, got, 0);
        end = base + kGrab;
    }
}

// y = A x, one warp per row, no atomics; y is cleared beforehand, rows
// without a hull path are skipped.
__global__ void __launch_bounds__(kWarpCta, kWarpCtaMin)
k_forward(GridC g, MlpC mc, RecView rv, const uint8_t* __restrict__ mask, unsigned* flags,
          int64_t n, const float* __restrict__ x, float* __restrict__ y, unsigned long long* next,
          int first)
{
    extern __shared__ unsigned char smem[];
    for_each_item(n, first, next, [&](int64_t i) {
        Path P;
        if (!load_path(rv, i, mc, P)) return;
        LaneWalk w;
        float s, q;
        warp_walk<0, true>(P, mc, g, mask, x, flags, warp_slots(smem, 0), mc.cmin, w, s, q);
        if ((threadIdx.x & 31) == 0) y[i] = s;
    });
}

// g = A^T y, one warp per row, scatter by FP32 atomics.
__global__ void __launch_bounds__(kWarpCta, kWarpCtaMin)
k_adjoint(GridC g, MlpC mc, RecView rv, const uint8_t* __restrict__ mask, unsigned* flags,
          int64_t n, const float* __restrict__ y, float* gout, unsigned long long* next, int first)
{
    extern __shared__ unsigned char smem[];
    const RunSlots slots = warp_slots(smem, kRunSlots);
    for_each_item(n, first, next, [&](int64_t i) {
        const float yi = __ldg(y + i);
        if (yi == 0.f) return;
        Path P;
        if (!load_path(rv, i, mc, P)) return;
        LaneWalk w;
        float s, q;
        warp_walk<kRunSlots, false>(P, mc, g, mask, nullptr, flags, slots, mc.cmin, w, s, q);
        replay_runs<kRunSlots>(P, mc, g, mask, flags, slots, w,
                               [&](int j, float l) { atomicAdd(gout + j, l * yi); });
    });
}

// DROP block step (Sec. IV-B; MLP, walk, row dot and scatter fused), one warp
// per proton of the block, x frozen:
//   r_i = (b_i - a_i.x) / ||a_i||^2, then acc[j] += (a_ij r_i, 1) over its row.
// The row is walked once; the scatter replays the runs kept in shared memory.
// The block's protons are the entries vidx[boff[k] .. boff[k+1]) of the list
// of protons whose path crosses the hull (the others have empty rows).
__global__ void __launch_bounds__(kWarpCta, kWarpCtaMin)
k_drop_fused(GridC g, MlpC mc, RecView rv, const uint8_t* __restrict__ mask, unsigned* flags,
             const int64_t* __restrict__ vidx, const int64_t* __restrict__ boff, int64_t k,
             const float* __restrict__ x, float2* acc, unsigned long long* next, int first)
{
    extern __shared__ unsigned char smem[];
    const RunSlots slots = warp_slots(smem, kRunSlots);
    const int64_t lo = boff[k];
    for_each_item(boff[k + 1] - lo, first, next, [&](int64_t t) {
        const int64_t i = vidx[lo + t];
        Path P;
        if (!load_path(rv, i, mc, P)) return;
        LaneWalk w;
        float s, q;
        warp_walk<kRunSlots, true>(P, mc, g, mask, x, flags, slots, mc.cmin, w, s, q);
        if (!(q > 0.f)) return;
        const float r = (rv.get(R_B, i) - s) / q;
        replay_runs<kRunSlots>(P, mc, g, mask, flags, slots, w,
                               [&](int j, float l) { atomicAdd(acc + j, make_float2(l * r, 1.f)); });
    });
}

// The same DROP block step with the round walk (pct_round.cuh): the row is
// built into the warp's run list, then s = a_i.x and q = ||a_i||^2 are gathered
// and the scatter is issued lane-strided over the list.  A proton that does
// not fit the round walk takes the lane-range walk (same shared memory).
static_assert(kRoundRuns * 8 == kRunSlots * kWarp * 8, "run list and run slots share a warp's shared memory");

// The lane-range DROP step of one proton, for the protons the round walk does
// not fit; not inlined, so that its registers do not weigh on the round walk.
__device__ __noinline__ void drop_proton_lanes(const Path& P, const MlpC& mc, const GridC& g,
                                               const uint8_t* __restrict__ mask, unsigned* flags, RunSlots slots,
                                               const float* __restrict__ x, float b, float2* acc)
{
    LaneWalk w;
    float s, q;
    warp_walk<kRunSlots, true>(P, mc, g, mask, x, flags, slots, mc.cmin, w, s, q);
    if (!(q > 0.f)) return;
    const float r = (b - s) / q;
    replay_runs<kRunSlots>(P, mc, g, mask, flags, slots, w,
                           [&](int j, float l) { atomicAdd(acc + j, make_float2(l * r, 1.f)); });
}

__global__ void __launch_bounds__(kWarpCta, kWarpCtaMin)
k_drop_rounds(GridC g, MlpC mc, RecView rv, const uint8_t* __restrict__ mask, unsigned* flags,
              const int64_t* __restrict__ vidx, const int64_t* __restrict__ boff, int64_t k,
              const float* __restrict__ x, float2* acc, unsigned long long* next, int first,
              unsigned long long* fallbacks)
{
    extern __shared__ unsigned char smem[];
    const RunSlots slots = warp_slots(smem, kRunSlots);
    const RunList list = warp_list(smem, kRunSlots);
    const int lane = threadIdx.x & (kWarp - 1);
    const int64_t lo = boff[k];
    for_each_item(boff[k + 1] - lo, first, next, [&](int64_t t) {
        const int64_t i = vidx[lo + t];
        Path P;
        if (!load_path(rv, i, mc, P)) return;
        int total = 0;
        if (round_runs(P, mc, g, list, total)) {
            float s = 0.f, q = 0.f;
            for (int e = lane; e < total; e += kWarp) {
                int j = list.j[e];
                const float l = list.l[e];
                if (j >= 0) {
                    if (__ldg(mask + j)) {
                        s = fmaf(l, __ldg(x + j), s);
                        q = fmaf(l, l, q);
                    } else {
                        j = -1;
                    }
                }
                list.j[e] = j;   // the hull decision, for the scatter below
            }
#pragma unroll
            for (int o = kWarp / 2; o > 0; o >>= 1) {
                s += __shfl_xor_sync(0xffffffffu, s, o);
                q += __shfl_xor_sync(0xffffffffu, q, o);
            }
            if (q > 0.f) {
                const float r = (rv.get(R_B, i) - s) / q;
                for (int e = lane; e < total; e += kWarp) {
                    const int j = list.j[e];
                    if (j >= 0) atomicAdd(acc + j, make_float2(list.l[e] * r, 1.f));
                }
            }
            __syncwarp();
            return;
        }
        if (fallbacks && lane == 0) atomicAdd(fallbacks, 1ull);
        drop_proton_lanes(P, mc, g, mask, flags, slots, x, rv.get(R_B, i), acc);
        __syncwarp();
    });
}

// Rows of A in path order with the round walk (debug / parity): what
// k_drop_rounds scatters.  Two warps per CTA; a proton that does not fit the
// round walk takes the lane-range walk of k_rows.
__global__ void __launch_bounds__(64)
k_rows_rounds(GridC g, MlpC mc, RecView rv, const uint8_t* __restrict__ mask, unsigned* flags,
              int64_t first, int64_t count, int32_t max_nnz, int32_t* __restrict__ idx,
              float* __restrict__ len, int32_t* __restrict__ nnz)
{
    extern __shared__ unsigned char smem[];
    const int lane = threadIdx.x & (kWarp - 1);
    const int64_t t = blockIdx.x * (int64_t)(blockDim.x >> 5) + (threadIdx.x >> 5);
    if (t >= count) return;
    Path P;
    if (!load_path(rv, first + t, mc, P)) {
        if (lane == 0) nnz[t] = 0;
        return;
    }
    const RunSlots slots = warp_slots(smem, kRowSlots);
    const RunList list = warp_list(smem, kRowSlots);
    int32_t* oi = idx + t * (int64_t)max_nnz;
    float* ol = len + t * (int64_t)max_nnz;
    int total = 0;
    if (round_runs(P, mc, g, list, total)) {
        if (lane == 0) {
            int n = 0;
            for (int e = 0; e < total; ++e) {
                const int j = list.j[e];
                if (j < 0 || !__ldg(mask + j)) continue;
                if (n < max_nnz) {
                    oi[n] = j;
                    ol[n] = list.l[e];
                }
                ++n;
            }
            nnz[t] = n;
        }
        return;
    }
    LaneWalk w;
    float s, q;
    warp_walk<kRowSlots, false>(P, mc, g, mask, nullptr, flags, slots, mc.cmin, w, s, q);
    if (__any_sync(0xffffffffu, w.n > kRowSlots)) {
        if (lane == 0) {
            nnz[t] = -1;
            atomicOr(flags, kFlagRowSlots);
        }
        return;
    }
    int mine = (w.k0 < w.k1) ? w.n - ((w.merged_prev && w.head_in) ? 1 : 0) : 0;
    int off = mine;
#pragma unroll
    for (int o = 1; o < kWarp; o <<= 1) {
        const int v = __shfl_up_sync(0xffffffffu, off, o);
        if (lane >= o) off += v;
    }
    const int tot = __shfl_sync(0xffffffffu, off, kWarp - 1);
    off -= mine;
    replay_runs<kRowSlots>(P, mc, g, mask, flags, slots, w, [&](int j, float l) {
        if (off < max_nnz) {
            oi[off] = j;
            ol[off] = l;
        }
        ++off;
    });
    if (lane == 0) nnz[t] = tot;
}

// DROP block apply (Sec. IV-B): x_j += lambda * num_j / s_j where the block touched
// voxel j, and clear the accumulator for the next block.
// `next` (if not null): the work counter of the block step, reset here for
// the next block step on the stream.
// Block apply, 4 voxels per group: the hull bytes of two groups are read
// first, then the accumulator and x of the groups that hold a hull voxel (the
// others are never scattered into, and whole 32-byte sectors of their
// accumulator are skipped).  x must be 16-byte aligned; k_drop_apply takes
// the voxels from 4 * n4 on, and every voxel when x is not aligned.
__device__ __forceinline__ void apply_group(uchar4 m, float4* __restrict__ x4, float4* __restrict__ acc4,
                                            int64_t g, float lambda)
{
    float4 a01 = acc4[2 * g], a23 = acc4[2 * g + 1];
    if (!((m.x && a01.y > 0.f) || (m.y && a01.w > 0.f) || (m.z && a23.y > 0.f) || (m.w && a23.w > 0.f)))
        return;
    float4 xv = x4[g];
    if (m.x && a01.y > 0.f) { xv.x = fmaf(lambda, a01.x / a01.y, xv.x); a01.x = a01.y = 0.f; }
    if (m.y && a01.w > 0.f) { xv.y = fmaf(lambda, a01.z / a01.w, xv.y); a01.z = a01.w = 0.f; }
    if (m.z && a23.y > 0.f) { xv.z = fmaf(lambda, a23.x / a23.y, xv.z); a23.x = a23.y = 0.f; }
    if (m.w && a23.w > 0.f) { xv.w = fmaf(lambda, a23.z / a23.w, xv.w); a23.z = a23.w = 0.f; }
    x4[g] = xv;
    acc4[2 * g] = a01;
    acc4[2 * g + 1] = a23;
}

__global__ void k_drop_apply4(int64_t n4, const uchar4* __restrict__ mask4, float4* __restrict__ x4,
                              float4* __restrict__ acc4, float lambda, unsigned long long* next)
{
    if (next && blockIdx.x == 0 && threadIdx.x == 0) *next = 0ull;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    for (; g + stride < n4; g += 2 * stride) {
        const uchar4 m0 = __ldg(mask4 + g), m1 = __ldg(mask4 + g + stride);
        const bool h0 = m0.x | m0.y | m0.z | m0.w, h1 = m1.x | m1.y | m1.z | m1.w;
        if (h0) apply_group(m0, x4, acc4, g, lambda);
        if (h1) apply_group(m1, x4, acc4, g + stride, lambda);
    }
    if (g < n4) {
        const uchar4 m0 = __ldg(mask4 + g);
        if (m0.x | m0.y | m0.z | m0.w) apply_group(m0, x4, acc4, g, lambda);
    }
}

__global__ void k_drop_apply(int64_t first, int64_t n_vox, const uint8_t* __restrict__ mask,
                             float* __restrict__ x, float2* __restrict__ acc, float lambda,
                             unsigned long long* next)
{
    if (next && blockIdx.x == 0 && threadIdx.x == 0) *next = 0ull;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t j = first + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < n_vox; j += stride) {
        if (!__ldg(mask + j)) continue;   // never scattered into
        const float2 a = acc[j];
        if (a.y > 0.f) {
            x[j] = fmaf(lambda, a.x / a.y, x[j]);
            acc[j] = make_float2(0.f, 0.f);
        }
    }
}

}  // namespace

#define PCT_LAUNCH_TAIL(L) \
    do {                   \
        ++*(L).launches;   \
        return cudaGetLastError(); \
    } while (0)

cudaError_t launch_prepare_range(const Launch& L, const Geo& G, const float* hist, int64_t stride,
                                 int64_t first, int64_t count, float* rec)
{
    if (count <= 0) return cudaSuccess;
    const float diag = sqrtf((float)G.g.nx * G.g.dx * (float)G.g.nx * G.g.dx +
                             (float)G.g.ny * G.g.dy * (float)G.g.ny * G.g.dy +
                             (float)G.g.nz * G.g.dz * (float)G.g.nz * G.g.dz);
    const float Lmax = fminf(diag * 1.0001f + 1e-3f, (float)(G.mc.kmax - 2) * G.mc.du_mm);
    k_prepare<<<grid_for(count, L.cta), L.cta, 0, L.stream>>>(G.g, G.mask, G.dist, G.flags, hist, stride,
                                                              first, count, rec, Lmax);
    PCT_LAUNCH_TAIL(L);
}

cudaError_t launch_tan_angle(const Launch& L, const double* t, double* out, int64_t n)
{
    if (n <= 0) return cudaSuccess;
    k_tan_angle<<<grid_for(n, 256), 256, 0, L.stream>>>(t, out, n);
    PCT_LAUNCH_TAIL(L);
}

cudaError_t launch_prepare(const Launch& L, const Geo& G, const float* hist, int64_t stride,
                           int64_t n, float* rec)
{
    return launch_prepare_range(L, G, hist, stride, 0, n, rec);
}

cudaError_t launch_hull_dist(const Launch& L, const uint8_t* mask, int nx, int ny, int nz, uint8_t* tmp,
                             uint8_t* dist)
{
    const int64_t n_vox = (int64_t)nx * ny * nz;
    if (n_vox <= 0) return cudaSuccess;
    const int64_t rows = (int64_t)ny * nz;
    k_hull_dist_x<<<(unsigned)((rows + 255) / 256), 256, 0, L.stream>>>(mask, nx, rows, dist);
    const unsigned blocks = (unsigned)((n_vox + 255) / 256);
    k_hull_dist_axis<<<blocks, 256, 0, L.stream>>>(dist, ny, nx, n_vox, tmp);
    k_hull_dist_axis<<<blocks, 256, 0, L.stream>>>(tmp, nz, (int64_t)nx * ny, n_vox, dist);
    *L.launches += 3;
    return cudaGetLastError();
}

cudaError_t launch_hull_states(const Launch& L, const float* rec, int64_t stride, int64_t first,
                               int64_t count, float* out)
{
    if (count <= 0) return cudaSuccess;
    k_hull_states<<<grid_for(count, L.cta), L.cta, 0, L.stream>>>(rec, stride, first, count, out);
    PCT_LAUNCH_TAIL(L);
}

cudaError_t launch_mlp_points(const Launch& L, const Geo& G, const float* rec, int64_t stride,
                              int64_t first, int64_t count, int32_t max_pts, float* out_xyz,
                              int32_t* out_npts)
{
    if (count <= 0) return cudaSuccess;
    k_mlp_points<<<grid_for(count, L.cta), L.cta, 0, L.stream>>>(
        G.g, G.mc, RecView{rec, stride}, first, count, max_pts, out_xyz, out_npts);
    PCT_LAUNCH_TAIL(L);
}

inline unsigned warp_grid(int64_t n, int cta)
{
    const int wpc = cta / kWarp;
    return (unsigned)((n + wpc - 1) / wpc);
}

inline size_t slot_bytes(int cta, int rl)
{
    return (size_t)(cta / kWarp) * rl * kWarp * 8;
}

template <class K>
cudaError_t allow_smem(K kernel, size_t bytes)
{
    if (bytes <= 48 * 1024) return cudaSuccess;
    return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

cudaError_t launch_rows(const Launch& L, const Geo& G, const float* rec, int64_t stride,
                        int64_t first, int64_t count, int32_t max_nnz, int32_t* out_idx,
                        float* out_len, int32_t* out_nnz)
{
    if (count <= 0) return cudaSuccess;
    const int cta = 64;   // 2 warps: the row writer keeps 64 slots per lane
    const size_t sm = slot_bytes(cta, kRowSlots);
    const auto kern = G.walk == kWalkRounds ? k_rows_rounds : k_rows;
    cudaError_t e = allow_smem(kern, sm);
    if (e != cudaSuccess) return e;
    kern<<<warp_grid(count, cta), cta, sm, L.stream>>>(G.g, G.mc, RecView{rec, stride}, G.mask, G.flags, first,
                                                       count, max_nnz, out_idx, out_len, out_nnz);
    PCT_LAUNCH_TAIL(L);
}

// Launch shape of a warp-per-item kernel over `count` items: one warp per item
// up to the CTAs that fill the GPU once (resident CTAs per SM x SMs, cached
// per thread, device and CTA size), and the first chunk per warp.
template <class K>
cudaError_t item_shape(K kernel, int cta, size_t smem, int64_t count, unsigned& grid, int& first)
{
    thread_local const void* fill_kernel = nullptr;
    thread_local int fill_dev = -1, fill_cta = -1, fill = 0;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (fill_kernel != (const void*)kernel || fill_dev != dev || fill_cta != cta) {
        int per_sm = 0, sms = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, cta, smem);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (e != cudaSuccess) return e;
        fill = per_sm * sms;
        fill_kernel = (const void*)kernel;
        fill_dev = dev;
        fill_cta = cta;
    }
    grid = warp_grid(count, cta);
    if (fill > 0 && grid > (unsigned)fill) grid = (unsigned)fill;
    const int64_t warps = (int64_t)grid * (cta / kWarp);
    first = count >= (int64_t)kGrab * warps ? kGrab : 1;
    return cudaSuccess;
}

cudaError_t launch_forward(const Launch& L, const Geo& G, const float* rec, int64_t stride,
                           int64_t n, const float* x, float* y, unsigned long long* next)
{
    if (n <= 0) return cudaSuccess;
    unsigned grid;
    int first;
    cudaError_t e = item_shape(k_forward, L.cta, 0, n, grid, first);
    if (e == cudaSuccess) e = cudaMemsetAsync(y, 0, (size_t)n * sizeof(float), L.stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(next, 0, sizeof(unsigned long long), L.stream);
    if (e != cudaSuccess) return e;
    k_forward<<<grid, L.cta, 0, L.stream>>>(G.g, G.mc, RecView{rec, stride}, G.mask, G.flags, n, x, y,
                                            next, first);
    PCT_LAUNCH_TAIL(L);
}

cudaError_t launch_adjoint(const Launch& L, const Geo& G, const float* rec, int64_t stride,
                           int64_t n, const float* y, float* g_out, unsigned long long* next)
{
    if (n <= 0) return cudaSuccess;
    const size_t sm = slot_bytes(L.cta, kRunSlots);
    cudaError_t e = allow_smem(k_adjoint, sm);
    unsigned grid;
    int first;
    if (e == cudaSuccess) e = item_shape(k_adjoint, L.cta, sm, n, grid, first);
    if (e == cudaSuccess) e = cudaMemsetAsync(next, 0, sizeof(unsigned long long), L.stream);
    if (e != cudaSuccess) return e;
    k_adjoint<<<grid, L.cta, sm, L.stream>>>(G.g, G.mc, RecView{rec, stride}, G.mask, G.flags, n, y,
                                             g_out, next, first);
    PCT_LAUNCH_TAIL(L);
}

cudaError_t launch_drop_fused(const Launch& L, const Geo& G, const float* rec, int64_t stride,
                              const int64_t* vidx, const int64_t* boff, int64_t k, int64_t count,
                              const float* x, float2* acc, unsigned long long* next)
{
    if (count <= 0) return cudaSuccess;
    const size_t sm = slot_bytes(L.cta, kRunSlots);
    unsigned grid;
    int first;
    cudaError_t e;
    if (G.walk == kWalkRounds) {
        e = allow_smem(k_drop_rounds, sm);
        if (e == cudaSuccess) e = item_shape(k_drop_rounds, L.cta, sm, count, grid, first);
        if (e != cudaSuccess) return e;
        k_drop_rounds<<<grid, L.cta, sm, L.stream>>>(G.g, G.mc, RecView{rec, stride}, G.mask, G.flags, vidx, boff,
                                                     k, x, acc, next, first, G.fallbacks);
    } else {
        e = allow_smem(k_drop_fused, sm);
        if (e == cudaSuccess) e = item_shape(k_drop_fused, L.cta, sm, count, grid, first);
        if (e != cudaSuccess) return e;
        k_drop_fused<<<grid, L.cta, sm, L.stream>>>(G.g, G.mc, RecView{rec, stride}, G.mask, G.flags, vidx, boff,
                                                    k, x, acc, next, first);
    }
    PCT_LAUNCH_TAIL(L);
}

// ---------------------------------------------------------------------------
// Valid-proton lists of the DROP blocks.  Three passes over the records:
// count the protons with a hull path (L > 0) per chunk, scan the chunk counts,
// and write each valid proton's index at its exclusive prefix (so the list
// keeps proton order and every block's protons stay together); the prefix at
// each block start is the block's offset in the list.
// ---------------------------------------------------------------------------
constexpr int kCompactCta = 256;
constexpr int kCompactRounds = (int)(kCompactChunk / kCompactCta);
static_assert(kCompactChunk % kCompactCta == 0, "compaction chunk must be whole CTA rounds");
constexpr int kCompactScanCta = 1024;

__device__ __forceinline__ bool has_path(const float* __restrict__ rec, int64_t stride, int64_t n, int64_t i)
{
    return i < n && rec[R_L * stride + i] > 0.f;
}

__global__ void __launch_bounds__(kCompactCta)
k_compact_count(const float* __restrict__ rec, int64_t stride, int64_t n, int64_t* __restrict__ chunk_count)
{
    __shared__ int part[kCompactCta / 32];
    const int64_t base = blockIdx.x * kCompactChunk;
    int c = 0;
    for (int r = 0; r < kCompactRounds; ++r) c += has_path(rec, stride, n, base + r * kCompactCta + threadIdx.x);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
    if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = c;
    __syncthreads();
    if (threadIdx.x == 0) {
        int64_t t = 0;
        for (int w = 0; w < kCompactCta / 32; ++w) t += part[w];
        chunk_count[blockIdx.x] = t;
    }
}

// One CTA: exclusive scan of the chunk counts in place; the total goes to
// boff[nblocks].
__global__ void __launch_bounds__(kCompactScanCta)
k_compact_scan(int64_t* __restrict__ chunk, int64_t nchunks, int64_t* __restrict__ boff, int64_t nblocks)
{
    __shared__ int64_t part[kCompactScanCta];
    const int64_t per = (nchunks + kCompactScanCta - 1) / kCompactScanCta;
    const int64_t a = threadIdx.x * per, b = a + per < nchunks ? a + per : nchunks;
    int64_t sum = 0;
    for (int64_t c = a; c < b; ++c) sum += chunk[c];
    part[threadIdx.x] = sum;
    __syncthreads();
    // Hillis-Steele inclusive scan of the per-thread sums
    for (int o = 1; o < kCompactScanCta; o <<= 1) {
        const int64_t v = threadIdx.x >= o ? part[threadIdx.x - o] : 0;
        __syncthreads();
        part[threadIdx.x] += v;
        __syncthreads();
    }
    int64_t run = part[threadIdx.x] - sum;
    for (int64_t c = a; c < b; ++c) {
        const int64_t v = chunk[c];
        chunk[c] = run;
        run += v;
    }
    if (threadIdx.x == kCompactScanCta - 1) boff[nblocks] = part[threadIdx.x];
}

__global__ void __launch_bounds__(kCompactCta)
k_compact_fill(const float* __restrict__ rec, int64_t stride, int64_t n, int64_t B,
               const int64_t* __restrict__ chunk_off, int64_t* __restrict__ vidx, int64_t* __restrict__ boff)
{
    __shared__ int part[kCompactCta / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t base = blockIdx.x * kCompactChunk;
    int64_t run = chunk_off[blockIdx.x];
    for (int r = 0; r < kCompactRounds; ++r) {
        const int64_t i = base + r * kCompactCta + threadIdx.x;
        const bool v = has_path(rec, stride, n, i);
        const unsigned bal = __ballot_sync(0xffffffffu, v);
        if (lane == 0) part[warp] = __popc(bal);
        __syncthreads();
        int before = 0, total = 0;
        for (int w = 0; w < kCompactCta / 32; ++w) {
            before += w < warp ? part[w] : 0;
            total += part[w];
        }
        const int64_t pos = run + before + __popc(bal & ((1u << lane) - 1u));
        if (i < n && i % B == 0) boff[i / B] = pos;
        if (v) vidx[pos] = i;
        run += total;
        __syncthreads();
    }
}

int64_t compact_chunks(int64_t n)
{
    return (n + kCompactChunk - 1) / kCompactChunk;
}

cudaError_t launch_compact(const Launch& L, const float* rec, int64_t stride, int64_t n, int64_t B,
                           int64_t* chunk, int64_t* vidx, int64_t* boff)
{
    if (n <= 0 || B <= 0) return cudaSuccess;
    const int64_t nc = compact_chunks(n), nblocks = (n + B - 1) / B;
    k_compact_count<<<(unsigned)nc, kCompactCta, 0, L.stream>>>(rec, stride, n, chunk);
    k_compact_scan<<<1, kCompactScanCta, 0, L.stream>>>(chunk, nc, boff, nblocks);
    k_compact_fill<<<(unsigned)nc, kCompactCta, 0, L.stream>>>(rec, stride, n, B, chunk, vidx, boff);
    *L.launches += 3;
    return cudaGetLastError();
}

cudaError_t launch_drop_apply(const Launch& L, int64_t n_vox, const uint8_t* mask, float* x, float2* acc,
                              float lambda, unsigned long long* next)
{
    if (n_vox <= 0) return cudaSuccess;
    // the mask and the accumulator are the library's own allocations
    // (256-byte aligned); x is the caller's
    const bool vec = ((uintptr_t)x & 15u) == 0 && ((uintptr_t)mask & 3u) == 0 && ((uintptr_t)acc & 15u) == 0;
    const int64_t n4 = vec ? n_vox / 4 : 0;
    if (n4 > 0) {
        int64_t blocks = (n4 + 255) / 256;
        if (blocks > 148 * 8) blocks = 148 * 8;
        k_drop_apply4<<<(unsigned)blocks, 256, 0, L.stream>>>(n4, (const uchar4*)mask, (float4*)x, (float4*)acc,
                                                              lambda, next);
        ++*L.launches;
        if (cudaError_t e = cudaGetLastError()) return e;
        if (4 * n4 == n_vox) return cudaSuccess;
        next = nullptr;
    }
    const int64_t rest = n_vox - 4 * n4;
    int64_t blocks = (rest + 255) / 256;
    if (blocks > 148 * 16) blocks = 148 * 16;
    k_drop_apply<<<(unsigned)blocks, 256, 0, L.stream>>>(4 * n4, n_vox, mask, x, acc, lambda, next);
    PCT_LAUNCH_TAIL(L);
}

}  // namespace pct
