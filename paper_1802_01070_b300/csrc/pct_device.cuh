// pct_device.cuh -- device-side building blocks of libpct (sm_103a).
//
// One proton is one thread (arXiv:1802.01070, Sec. I).  For each proton the
// hot path recomputes, with no storage of A:
//   1. its most likely path (MLP) at depths u_in + k*du, from the hull-frame
//      entry/exit states (Gaussian multiple-scattering MLP cited in Sec. I);
//   2. a 3D voxel walk along the MLP polyline, producing the row a_i as a
//      sequence of (voxel j, chord a_ij) visits;
// (pct_warp.cuh), one warp per proton.
//
// MLP arithmetic here (FP32, Kalman form):
//   y1 = R0 y0 + S1 R1^T (R1 S1 R1^T + S2)^-1 (y2 - R1 R0 y0),
// algebraically the same state as the information form of the method; only
// the position row is needed for the walk.  S1 = Sigma(0, w) depends on the
// sample index alone and is read from a per-context table; S2 = Sigma(w, L)
// uses the moments of 1/(beta^2 p^2) Taylor-shifted to the exit depth, so that
// no cancellation grows as w -> L.
#pragma once

#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

namespace pct {

// Highland multiple-scattering constants for water.
constexpr float kE0 = 13.6f;   // MeV
constexpr float kX0 = 36.08f;  // cm

// Device-flag bits (context error word).
constexpr unsigned kFlagWalkGuard = 1u;   // a segment walk exceeded its step bound
constexpr unsigned kFlagHullGuard = 2u;   // a hull search exceeded its step bound
constexpr unsigned kFlagMlpTable = 4u;    // MLP sample index beyond the S1 table
constexpr unsigned kFlagRowSlots = 8u;    // a debug row had more runs per lane than its slots
constexpr unsigned kFlagPackStep = 16u;   // packed rows: consecutive runs not in neighbouring voxels
constexpr unsigned kFlagRowBounds = 32u;  // a stored row's length or voxel index out of range
constexpr unsigned kFlagChordRange = 128u; // packed rows: a chord beyond the fixed-point range (clamped)
constexpr unsigned kFlagBarrierTimeout = 64u;  // a bounded barrier wait gave up

struct GridC {
    int nx, ny, nz;
    float dx, dy, dz;
    float ox, oy, oz;
    float idx, idy, idz;  // 1 / voxel edge
};

struct MlpC {
    float du_mm, du_cm, dend_mm;
    float coef[6];        // 1/(beta^2 p^2) = sum coef[k] u^k, MeV^-2, u in cm
    const float4* sig1;   // sig1[k] = Sigma(0, k*du): (S00, S01, S11, 2 S01), cm / rad
    int kmax;             // last valid index of sig1
    int cmin;             // fewest segments per lane range whose depth exceeds a voxel diagonal
};

// Per-proton record written once per call by the prepare kernel (SoA).
enum RecField {
    R_C = 0, R_S,           // cos, sin of the gantry angle
    R_UIN, R_L,             // hull entry depth (mm) and path depth L = u_out - u_in (0: empty row)
    R_T0, R_TH0, R_V0, R_PS0,
    R_T2, R_TH2, R_V2, R_PS2,
    R_PX, R_PY, R_PZ,       // hull entry point in grid units ((p - o) / d)
    R_B,                    // WEPL, mm
    R_NF
};

struct RecView {
    const float* p;
    int64_t stride;
    __device__ __forceinline__ float get(int f, int64_t i) const { return __ldg(p + f * stride + i); }
};

// Register-resident description of one proton's path.
struct Path {
    float c, s;
    float L_mm, L_cm;
    float th0, ps0;
    float d0t, d1t, d0v, d1v;  // y2 - R(L) y0 per plane: position (mm) and angle (rad)
    float dt, dv;              // exit point offsets t2 - t0, v2 - v0 (mm)
    float px, py, pz;          // entry point, grid units
    float c2[6];               // f(L - w) = sum c2[m] w^m (w in cm)
    int nseg;                  // polyline segments
};

__device__ __forceinline__ bool load_path(const RecView& r, int64_t i, const MlpC& mc, Path& P)
{
    P.L_mm = r.get(R_L, i);
    if (!(P.L_mm > 0.f)) return false;
    P.c = r.get(R_C, i);
    P.s = r.get(R_S, i);
    P.th0 = r.get(R_TH0, i);
    P.ps0 = r.get(R_PS0, i);
    P.dt = r.get(R_T2, i) - r.get(R_T0, i);
    P.dv = r.get(R_V2, i) - r.get(R_V0, i);
    P.d0t = P.dt - P.L_mm * P.th0;
    P.d1t = r.get(R_TH2, i) - P.th0;
    P.d0v = P.dv - P.L_mm * P.ps0;
    P.d1v = r.get(R_PS2, i) - P.ps0;
    P.px = r.get(R_PX, i);
    P.py = r.get(R_PY, i);
    P.pz = r.get(R_PZ, i);
    P.L_cm = 0.1f * P.L_mm;
    // Taylor shift of the depth polynomial to u = L: b[m] = f^(m)(L)/m!
    float b[6];
#pragma unroll
    for (int k = 0; k < 6; ++k) b[k] = mc.coef[k];
#pragma unroll
    for (int i2 = 0; i2 < 5; ++i2)
#pragma unroll
        for (int k = 4; k >= i2; --k) b[k] = fmaf(P.L_cm, b[k + 1], b[k]);
#pragma unroll
    for (int m = 0; m < 6; ++m) P.c2[m] = (m & 1) ? -b[m] : b[m];
    // interior samples k*du < L - dend, k >= 1
    float lim = P.L_mm - mc.dend_mm;
    int kin = lim > 0.f ? (int)ceilf(lim / mc.du_mm) - 1 : 0;
    if (kin < 0) kin = 0;
    P.nseg = kin + 1;
    return true;
}

// MLP position offsets (t, v relative to the entry state, mm) at sample k.
__device__ __forceinline__ void mlp_offset(const Path& P, const MlpC& mc, int k, float& w_mm,
                                           float& dt, float& dv)
{
    w_mm = (float)k * mc.du_mm;
    const float W = P.L_cm - (float)k * mc.du_cm;   // depth left to the exit, cm
    const float4 s1 = __ldg(mc.sig1 + k);
    // int_0^W w^n f(L - w) dw = W^(n+1) sum_m c2[m] W^m / (n+m+1), n = 0, 1, 2
    float q0 = P.c2[5] * (1.f / 6.f), q1 = P.c2[5] * (1.f / 7.f), q2 = P.c2[5] * (1.f / 8.f);
    q0 = fmaf(q0, W, P.c2[4] * (1.f / 5.f));
    q1 = fmaf(q1, W, P.c2[4] * (1.f / 6.f));
    q2 = fmaf(q2, W, P.c2[4] * (1.f / 7.f));
    q0 = fmaf(q0, W, P.c2[3] * (1.f / 4.f));
    q1 = fmaf(q1, W, P.c2[3] * (1.f / 5.f));
    q2 = fmaf(q2, W, P.c2[3] * (1.f / 6.f));
    q0 = fmaf(q0, W, P.c2[2] * (1.f / 3.f));
    q1 = fmaf(q1, W, P.c2[2] * (1.f / 4.f));
    q2 = fmaf(q2, W, P.c2[2] * (1.f / 5.f));
    q0 = fmaf(q0, W, P.c2[1] * (1.f / 2.f));
    q1 = fmaf(q1, W, P.c2[1] * (1.f / 3.f));
    q2 = fmaf(q2, W, P.c2[1] * (1.f / 4.f));
    q0 = fmaf(q0, W, P.c2[0]);
    q1 = fmaf(q1, W, P.c2[0] * (1.f / 2.f));
    q2 = fmaf(q2, W, P.c2[0] * (1.f / 3.f));
    // Highland factor: an absolute error of 1e-6 in the logarithm moves it by
    // 4e-8 relative, so the hardware log2 is accurate enough here
    const float lf = fmaf(0.038f * 0.69314718f, __log2f(W * (1.f / kX0)), 1.f);
    const float pre = (kE0 * kE0 / kX0) * lf * lf * W;
    const float T11 = pre * q0;             // Sigma2 entries (cm, rad)
    const float T01 = pre * W * q1;
    const float T00 = pre * W * W * q2;
    const float M00 = fmaf(W, fmaf(W, s1.z, s1.w), s1.x) + T00;
    const float M01 = fmaf(W, s1.z, s1.y) + T01;
    const float M11 = s1.z + T11;
    const float g0 = fmaf(W, s1.y, s1.x);
    const float g1 = s1.y;
    const float rdet = __fdividef(1.f, fmaf(M00, M11, -M01 * M01));
    const float G0 = fmaf(g0, M11, -g1 * M01) * rdet;           // dimensionless
    const float G1 = fmaf(g1, M00, -g0 * M01) * rdet * 10.f;    // mm per rad
    dt = fmaf(w_mm, P.th0, fmaf(G0, P.d0t, G1 * P.d1t));
    dv = fmaf(w_mm, P.ps0, fmaf(G0, P.d0v, G1 * P.d1v));
}

// Polyline vertex k (k = 0: hull entry, k = nseg: hull exit), grid units.
__device__ __forceinline__ void path_point(const Path& P, const MlpC& mc, const GridC& g, int k,
                                           float& x, float& y, float& z)
{
    float w, dt, dv;
    if (k <= 0) {
        x = P.px;
        y = P.py;
        z = P.pz;
        return;
    }
    if (k >= P.nseg) {
        w = P.L_mm;
        dt = P.dt;
        dv = P.dv;
    } else {
        mlp_offset(P, mc, k, w, dt, dv);
    }
    x = fmaf(fmaf(w, P.c, -dt * P.s), g.idx, P.px);
    y = fmaf(fmaf(w, P.s, dt * P.c), g.idy, P.py);
    z = fmaf(dv, g.idz, P.pz);
}

__device__ __forceinline__ int start_index(float a, float dir)
{
    float f = floorf(a);
    int k = (int)f;
    if (a == f && dir < 0.f) k -= 1;   // on a face: the voxel the path moves into
    return k;
}

__device__ __forceinline__ bool in_grid(const GridC& g, int ix, int iy, int iz)
{
    return (unsigned)ix < (unsigned)g.nx && (unsigned)iy < (unsigned)g.ny &&
           (unsigned)iz < (unsigned)g.nz;
}

// Linear voxel index (grids hold fewer than 2^31 voxels).
__device__ __forceinline__ int lin(const GridC& g, int ix, int iy, int iz)
{
    return ix + g.nx * (iy + g.ny * iz);
}

// ---------------------------------------------------------------------------
// Hull entry along a straight tracker line (reading: the paper names no hull
// rule; the path starts where the line first enters a hull voxel).
// Line p(s) = T + s D (grid units per mm of depth), s in [0, S].
// ---------------------------------------------------------------------------
// On a hit, (axis, face) name the grid plane the line crosses into the hull
// voxel (face in grid units along axis); axis = -1 when the line starts inside
// that voxel (s_hit = 0).  The caller re-evaluates the crossing parameter from
// them in FP64: for a line nearly parallel to the plane the FP32 parameter is
// ill-conditioned.
//
// Empty-space skipping: `dist` (optional) holds, per voxel, the chessboard
// distance d to the nearest hull voxel (0 inside the hull, capped at 255).
// Every voxel within chessboard distance d-1 of a voxel at distance d is
// outside the hull, so from a point of that voxel the line can advance until it
// has moved d-1 voxels along its dominant axis without passing a hull voxel.
// The jump keeps 1/16 voxel of slack for rounding and always ends in a voxel
// outside the hull, so the hull voxel is still entered by a DDA step that sets
// (axis, face).  Without `dist` the search visits every voxel.
__device__ __forceinline__ bool hull_entry(const GridC& g, const uint8_t* __restrict__ mask,
                                           const uint8_t* __restrict__ dist,
                                           float Tx, float Ty, float Tz, float Dx, float Dy,
                                           float Dz, float S, unsigned* flags, float& s_hit,
                                           int& axis, int& face)
{
    float s_lo = 0.f, s_hi = S;
    const float T[3] = {Tx, Ty, Tz};
    const float D[3] = {Dx, Dy, Dz};
    const int n[3] = {g.nx, g.ny, g.nz};
    axis = -1;
    face = 0;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        if (D[a] == 0.f) {
            if (T[a] < 0.f || T[a] >= (float)n[a]) return false;
        } else {
            float s1 = (0.f - T[a]) / D[a], s2 = ((float)n[a] - T[a]) / D[a];
            int f1 = 0;
            if (s1 > s2) {
                const float tmp = s1;
                s1 = s2;
                s2 = tmp;
                f1 = n[a];
            }
            if (s1 > s_lo) {
                s_lo = s1;
                axis = a;
                face = f1;
            }
            s_hi = fminf(s_hi, s2);
        }
    }
    if (!(s_lo < s_hi)) return false;
    int iv[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        int k = start_index(fmaf(s_lo, D[a], T[a]), D[a]);
        k = k < 0 ? 0 : (k > n[a] - 1 ? n[a] - 1 : k);
        iv[a] = k;
    }
    float s_cur = s_lo;
    const float inv_dmax = 1.f / fmaxf(fabsf(Dx), fmaxf(fabsf(Dy), fabsf(Dz)));
    const int guard = g.nx + g.ny + g.nz + 4;
    for (int it = 0; it <= guard; ++it) {
        const int j = lin(g, iv[0], iv[1], iv[2]);
        if (dist) {
            const int d = __ldg(dist + j);
            if (d == 0) {
                s_hit = s_cur;
                return true;
            }
            if (d >= 2) {
                const float s_jump = fmaf((float)d - 1.0625f, inv_dmax, s_cur);
                if (!(s_jump < s_hi)) return false;
                s_cur = s_jump;
#pragma unroll
                for (int a = 0; a < 3; ++a) {
                    int k = start_index(fmaf(s_jump, D[a], T[a]), D[a]);
                    iv[a] = k < 0 ? 0 : (k > n[a] - 1 ? n[a] - 1 : k);
                }
                continue;
            }
        } else if (__ldg(mask + j)) {
            s_hit = s_cur;
            return true;
        }
        float tm[3];
        float s_next = __int_as_float(0x7f800000);
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            if (D[a] > 0.f)
                tm[a] = ((float)(iv[a] + 1) - T[a]) / D[a];
            else if (D[a] < 0.f)
                tm[a] = ((float)iv[a] - T[a]) / D[a];
            else
                tm[a] = __int_as_float(0x7f800000);
            s_next = fminf(s_next, tm[a]);
        }
        if (!(s_next < s_hi)) return false;
#pragma unroll
        for (int a = 0; a < 3; ++a)
            if (tm[a] == s_next) {
                axis = a;
                face = D[a] > 0.f ? iv[a] + 1 : iv[a];
                iv[a] += D[a] > 0.f ? 1 : -1;
            }
        s_cur = s_next;
        if ((unsigned)iv[0] >= (unsigned)g.nx || (unsigned)iv[1] >= (unsigned)g.ny ||
            (unsigned)iv[2] >= (unsigned)g.nz)
            return false;
    }
    atomicOr(flags, kFlagHullGuard);
    return false;
}

}  // namespace pct
