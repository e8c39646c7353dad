// pct_kernels.cu -- CUDA kernels of libpct and their launchers (sm_103a).
//
// All per-proton kernels map one proton to one thread (arXiv:1802.01070,
// Sec. I) and recompute the proton's row of A from its record: MLP samples,
// then the voxel walk (pct_device.cuh).  None of them stores A.
#include "pct_internal.h"

namespace pct {

namespace {

constexpr int kMaxCta = 512;

inline unsigned grid_for(int64_t n, int cta)
{
    return (unsigned)((n + cta - 1) / cta);
}

// ---------------------------------------------------------------------------
// Hull-frame record of each proton (a2): rotate the tracker data into the
// beam frame of its gantry angle, follow both straight tracker lines to the
// hull, and store the entry/exit states the MLP starts from.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kMaxCta)
k_prepare(GridC g, const uint8_t* __restrict__ mask, unsigned* flags, const float* __restrict__ h,
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
    const float ua = fmaf(xi, c, yi * s), ta = fmaf(-xi, s, yi * c), va = zi;
    const float ub = fmaf(xo, c, yo * s), tb = fmaf(-xo, s, yo * c), vb = zo;
    const float tti = tanf(thi), tpi = tanf(psi), tto = tanf(tho), tpo = tanf(pso);
    bool ok = isfinite(ua) && isfinite(ub) && isfinite(ta) && isfinite(tb) && isfinite(va) &&
              isfinite(vb) && isfinite(tti) && isfinite(tpi) && isfinite(tto) && isfinite(tpo) &&
              ub > ua;
    const float S = ub - ua;
    // straight lines in grid units per mm of depth
    const float Tix = (xi - g.ox) * g.idx, Tiy = (yi - g.oy) * g.idy, Tiz = (zi - g.oz) * g.idz;
    const float Dix = fmaf(-tti, s, c) * g.idx, Diy = fmaf(tti, c, s) * g.idy, Diz = tpi * g.idz;
    const float Tox = (xo - g.ox) * g.idx, Toy = (yo - g.oy) * g.idy, Toz = (zo - g.oz) * g.idz;
    const float Dox = -fmaf(-tto, s, c) * g.idx, Doy = -fmaf(tto, c, s) * g.idy, Doz = -tpo * g.idz;
    float s_in = 0.f, s_out = 0.f;
    if (ok) ok = hull_entry(g, mask, Tix, Tiy, Tiz, Dix, Diy, Diz, S, flags, s_in);
    if (ok) ok = hull_entry(g, mask, Tox, Toy, Toz, Dox, Doy, Doz, S, flags, s_out);
    const float u_in = ua + s_in, u_out = ub - s_out;
    const float L = u_out - u_in;
    ok = ok && L > 0.f && L <= Lmax;
    rec[R_C * stride + i] = c;
    rec[R_S * stride + i] = s;
    rec[R_UIN * stride + i] = u_in;
    rec[R_L * stride + i] = ok ? L : 0.f;
    rec[R_T0 * stride + i] = fmaf(tti, s_in, ta);
    rec[R_TH0 * stride + i] = thi;
    rec[R_V0 * stride + i] = fmaf(tpi, s_in, va);
    rec[R_PS0 * stride + i] = psi;
    rec[R_T2 * stride + i] = fmaf(-tto, s_out, tb);
    rec[R_TH2 * stride + i] = tho;
    rec[R_V2 * stride + i] = fmaf(-tpo, s_out, vb);
    rec[R_PS2 * stride + i] = pso;
    rec[R_PX * stride + i] = fmaf(s_in, Dix, Tix);
    rec[R_PY * stride + i] = fmaf(s_in, Diy, Tiy);
    rec[R_PZ * stride + i] = fmaf(s_in, Diz, Tiz);
    rec[R_B * stride + i] = wepl;
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

// Rows of A in path order (debug / parity).
__global__ void __launch_bounds__(kMaxCta)
k_rows(GridC g, MlpC mc, RecView rv, const uint8_t* __restrict__ mask, unsigned* flags,
       int64_t first, int64_t count, int32_t max_nnz, int32_t* __restrict__ idx,
       float* __restrict__ len, int32_t* __restrict__ nnz)
{
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= count) return;
    Path P;
    if (!load_path(rv, first + t, mc, P)) {
        nnz[t] = 0;
        return;
    }
    RowWriter w{&g, mask, idx + (int64_t)t * max_nnz, len + (int64_t)t * max_nnz, max_nnz, 0};
    walk_path(P, mc, g, flags, w);
    nnz[t] = w.n;
}

// y = A x (a10): one row per thread, no atomics.
__global__ void __launch_bounds__(kMaxCta)
k_forward(GridC g, MlpC mc, RecView rv, const uint8_t* __restrict__ mask, unsigned* flags,
          int64_t n, const float* __restrict__ x, float* __restrict__ y)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    Path P;
    if (!load_path(rv, i, mc, P)) {
        y[i] = 0.f;
        return;
    }
    DotVisitor d{&g, mask, x, 0.f, 0.f, 0.f, 0.f, 0};
    walk_path(P, mc, g, flags, d);
    d.finish();
    y[i] = d.s;
}

// g = A^T y (a10): one row per thread, scatter by FP32 atomics.
__global__ void __launch_bounds__(kMaxCta)
k_adjoint(GridC g, MlpC mc, RecView rv, const uint8_t* __restrict__ mask, unsigned* flags,
          int64_t n, const float* __restrict__ y, float* gout)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    Path P;
    if (!load_path(rv, i, mc, P)) return;
    const float yi = y[i];
    if (yi == 0.f) return;
    AdjointVisitor a{&g, mask, gout, yi, 0, 0.f, 0};
    walk_path(P, mc, g, flags, a);
    a.finish();
}

// DROP block step (a3-a6 fused): per proton of the block, with x frozen,
//   r_i = (b_i - a_i.x) / ||a_i||^2, then acc[j] += (a_ij r_i, 1) on its row.
// The row is walked twice (dot, then scatter) instead of being stored.
__global__ void __launch_bounds__(kMaxCta)
k_drop_fused(GridC g, MlpC mc, RecView rv, const uint8_t* __restrict__ mask, unsigned* flags,
             int64_t first, int64_t count, const float* __restrict__ x, float2* acc)
{
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= count) return;
    const int64_t i = first + t;
    Path P;
    if (!load_path(rv, i, mc, P)) return;
    DotVisitor d{&g, mask, x, 0.f, 0.f, 0.f, 0.f, 0};
    walk_path(P, mc, g, flags, d);
    d.finish();
    if (!(d.q > 0.f)) return;
    const float r = (rv.get(R_B, i) - d.s) / d.q;
    ScatterVisitor sc{&g, mask, acc, r, 0, 0.f, 0};
    walk_path(P, mc, g, flags, sc);
    sc.finish();
}

// DROP block apply (a7): x_j += lambda * num_j / s_j where the block touched
// voxel j, and clear the accumulator for the next block.
__global__ void k_drop_apply(int64_t n_vox, float* __restrict__ x, float2* __restrict__ acc,
                             float lambda)
{
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < n_vox; j += stride) {
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

cudaError_t launch_prepare(const Launch& L, const Geo& G, const float* hist, int64_t stride,
                           int64_t n, float* rec)
{
    if (n <= 0) return cudaSuccess;
    const float diag = sqrtf((float)G.g.nx * G.g.dx * (float)G.g.nx * G.g.dx +
                             (float)G.g.ny * G.g.dy * (float)G.g.ny * G.g.dy +
                             (float)G.g.nz * G.g.dz * (float)G.g.nz * G.g.dz);
    const float Lmax = fminf(diag * 1.0001f + 1e-3f, (float)(G.mc.kmax - 2) * G.mc.du_mm);
    k_prepare<<<grid_for(n, L.cta), L.cta, 0, L.stream>>>(G.g, G.mask, G.flags, hist, stride, 0, n,
                                                          rec, Lmax);
    PCT_LAUNCH_TAIL(L);
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

cudaError_t launch_rows(const Launch& L, const Geo& G, const float* rec, int64_t stride,
                        int64_t first, int64_t count, int32_t max_nnz, int32_t* out_idx,
                        float* out_len, int32_t* out_nnz)
{
    if (count <= 0) return cudaSuccess;
    k_rows<<<grid_for(count, L.cta), L.cta, 0, L.stream>>>(G.g, G.mc, RecView{rec, stride}, G.mask,
                                                            G.flags, first, count, max_nnz, out_idx,
                                                            out_len, out_nnz);
    PCT_LAUNCH_TAIL(L);
}

cudaError_t launch_forward(const Launch& L, const Geo& G, const float* rec, int64_t stride,
                           int64_t n, const float* x, float* y)
{
    if (n <= 0) return cudaSuccess;
    k_forward<<<grid_for(n, L.cta), L.cta, 0, L.stream>>>(G.g, G.mc, RecView{rec, stride}, G.mask,
                                                          G.flags, n, x, y);
    PCT_LAUNCH_TAIL(L);
}

cudaError_t launch_adjoint(const Launch& L, const Geo& G, const float* rec, int64_t stride,
                           int64_t n, const float* y, float* g_out)
{
    if (n <= 0) return cudaSuccess;
    k_adjoint<<<grid_for(n, L.cta), L.cta, 0, L.stream>>>(G.g, G.mc, RecView{rec, stride}, G.mask,
                                                          G.flags, n, y, g_out);
    PCT_LAUNCH_TAIL(L);
}

cudaError_t launch_drop_fused(const Launch& L, const Geo& G, const float* rec, int64_t stride,
                              int64_t first, int64_t count, const float* x, float2* acc)
{
    if (count <= 0) return cudaSuccess;
    k_drop_fused<<<grid_for(count, L.cta), L.cta, 0, L.stream>>>(
        G.g, G.mc, RecView{rec, stride}, G.mask, G.flags, first, count, x, acc);
    PCT_LAUNCH_TAIL(L);
}

cudaError_t launch_drop_apply(const Launch& L, int64_t n_vox, float* x, float2* acc, float lambda)
{
    if (n_vox <= 0) return cudaSuccess;
    int64_t blocks = (n_vox + 255) / 256;
    if (blocks > 148 * 16) blocks = 148 * 16;
    k_drop_apply<<<(unsigned)blocks, 256, 0, L.stream>>>(n_vox, x, acc, lambda);
    PCT_LAUNCH_TAIL(L);
}

}  // namespace pct
