/*
 * pct_oracle.c -- plain, slow FP64 CPU oracle for the proton-CT hot path.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library links, calls or
 * includes this file; only tests/, the smoke check and the CPU-baseline leg of
 * bench.py load it.  It shares no code, header, table or constant with the
 * CUDA path: every constant below is written here independently.
 *
 * What it computes (Karbasi et al., "A Highly Accelerated Parallel Multi-GPU
 * based Reconstruction Algorithm ...", arXiv:1802.01070):
 *   - Sec. I: the linear model A x = b, A holding the path data of each
 *     proton, b the WEPLs and x the RSPs; each proton's path is its most
 *     likely path (MLP) from its tracker data.
 *   - Sec. IV-B: the block-iterative DROP solver, a block being the protons
 *     processed together.
 * The paper prints neither the MLP nor the DROP update, so this file follows
 * the published method it cites for each:
 *   - MLP (Schulte et al. 2008): Gaussian multiple-scattering prior, the
 *     scattering matrices Sigma1/Sigma2 as 2x2 moment integrals of
 *     1/(beta^2 p^2)(u), and the maximum-likelihood state
 *       y1 = (S1^-1 + R1^T S2^-1 R1)^-1 (S1^-1 R0 y0 + R1^T S2^-1 y2),
 *     evaluated here in this "information" form, FP64, per plane.
 *   - DROP (Penfold, Schulte, Censor et al. 2010): for each block of rows,
 *       x_j <- x_j + lambda / s_j * sum_i a_ij (b_i - <a_i,x>) / ||a_i||^2,
 *     s_j = number of rows of the block with a_ij > 0, x frozen during the
 *     block.
 * Readings where the paper is silent (hull rule, sample spacing, walk tie
 * rules) are stated next to the code that takes them.
 *
 * Parity status: every function is pinned by tests/test_oracle_pins.py against
 * closed forms, brute force or textbook special cases.  The whole
 * reconstruction is "parity unpinned" against the paper itself: the paper
 * prints no input data and no per-voxel values to compare with.
 *
 * Units: lab and beam frame positions in mm, angles in rad, scattering depth
 * in cm (the unit of the 1/(beta^2 p^2) polynomial).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

/* Highland/Lynch-Dahl multiple-scattering constants for water. */
#define O_E0_MEV 13.6
#define O_X0_CM 36.08

typedef struct {
    int32_t nx, ny, nz;
    int32_t highland;  /* 1: keep the logarithmic term of the Highland formula */
    double dx, dy, dz; /* voxel size, mm */
    double ox, oy, oz; /* grid corner, mm */
    double du;         /* MLP sample spacing along depth, mm */
    double dend;       /* no interior sample within dend (mm) of the exit depth */
    double coef[6];    /* 1/(beta^2 p^2) = sum coef[k] u^k, MeV^-2, u in cm */
} o_cfg;

/* ---------------------------------------------------------------------- */
/* Scattering matrices (Schulte et al. 2008, used by the paper's Sec. I)   */
/* ---------------------------------------------------------------------- */

static double o_poly(const double *c, double u)
{
    double acc = 0.0;
    for (int k = 5; k >= 0; --k) acc = acc * u + c[k];
    return acc;
}

/* 5-point Gauss-Legendre rule on [-1, 1]; exact for polynomials of degree <= 9.
 * The integrands below, (ub-u)^n * f(u) with n <= 2 and deg f = 5, have degree
 * <= 7, so the rule gives the integrals exactly up to rounding. */
static const double o_gl_x[5] = {-0.9061798459386640, -0.5384693101056831, 0.0,
                                 0.5384693101056831, 0.9061798459386640};
static const double o_gl_w[5] = {0.2369268850561891, 0.4786286704993665, 0.5688888888888889,
                                 0.4786286704993665, 0.2369268850561891};

/* Sigma(ua, ub) in cm/rad units:
 *   S[0] = P * int (ub-u)^2 f,  S[1] = P * int (ub-u) f,  S[2] = P * int f,
 * integrals over [ua, ub], P = E0^2 (1 + 0.038 ln((ub-ua)/X0))^2 / X0. */
int o_sigma(const o_cfg *cfg, double ua, double ub, double S[3])
{
    double h = ub - ua;
    if (!(h > 0.0)) {
        S[0] = S[1] = S[2] = 0.0;
        return 0;
    }
    double i0 = 0.0, i1 = 0.0, i2 = 0.0;
    for (int q = 0; q < 5; ++q) {
        double arm = 0.5 * h * (1.0 - o_gl_x[q]); /* ub - u at the node */
        double u = ub - arm;
        double fw = o_poly(cfg->coef, u) * 0.5 * h * o_gl_w[q];
        i0 += fw;
        i1 += arm * fw;
        i2 += arm * arm * fw;
    }
    double lf = cfg->highland ? (1.0 + 0.038 * log(h / O_X0_CM)) : 1.0;
    double pre = O_E0_MEV * O_E0_MEV * lf * lf / O_X0_CM;
    S[0] = pre * i2;
    S[1] = pre * i1;
    S[2] = pre * i0;
    return 0;
}

static int o_inv2(const double m[4], double out[4])
{
    double det = m[0] * m[3] - m[1] * m[2];
    if (det == 0.0 || !isfinite(det)) return -1;
    out[0] = m[3] / det;
    out[1] = -m[1] / det;
    out[2] = -m[2] / det;
    out[3] = m[0] / det;
    return 0;
}

static void o_mul2(const double a[4], const double b[4], double out[4])
{
    double r[4];
    r[0] = a[0] * b[0] + a[1] * b[2];
    r[1] = a[0] * b[1] + a[1] * b[3];
    r[2] = a[2] * b[0] + a[3] * b[2];
    r[3] = a[2] * b[1] + a[3] * b[3];
    memcpy(out, r, sizeof r);
}

static void o_mv2(const double a[4], const double v[2], double out[2])
{
    double r0 = a[0] * v[0] + a[1] * v[1];
    double r1 = a[2] * v[0] + a[3] * v[1];
    out[0] = r0;
    out[1] = r1;
}

/* MLP state (position cm, angle rad) at depth u1 in (0, L), entry state y0 at
 * depth 0 and exit state y2 at depth L (cm), information form. */
int o_mlp_point(const o_cfg *cfg, const double y0[2], const double y2[2], double L, double u1,
                double y1[2])
{
    double s1[3], s2[3];
    o_sigma(cfg, 0.0, u1, s1);
    o_sigma(cfg, u1, L, s2);
    double S1[4] = {s1[0], s1[1], s1[1], s1[2]};
    double S2[4] = {s2[0], s2[1], s2[1], s2[2]};
    double R0[4] = {1.0, u1, 0.0, 1.0};
    double R1[4] = {1.0, L - u1, 0.0, 1.0};
    double R1T[4] = {1.0, 0.0, L - u1, 1.0};
    double S1i[4], S2i[4];
    if (o_inv2(S1, S1i) || o_inv2(S2, S2i)) return -1;
    double t[4], H[4], Hi[4];
    o_mul2(R1T, S2i, t);  /* R1^T S2^-1 */
    o_mul2(t, R1, H);     /* R1^T S2^-1 R1 */
    for (int k = 0; k < 4; ++k) H[k] += S1i[k];
    if (o_inv2(H, Hi)) return -1;
    double a[2], c[2], rhs[2];
    o_mv2(R0, y0, a);
    o_mv2(S1i, a, a);     /* S1^-1 R0 y0 */
    o_mv2(t, y2, c);      /* R1^T S2^-1 y2 */
    rhs[0] = a[0] + c[0];
    rhs[1] = a[1] + c[1];
    o_mv2(Hi, rhs, y1);
    return 0;
}

/* ---------------------------------------------------------------------- */
/* Hull entry / exit (reading: not in the paper; first crossing into a     */
/* hull-mask voxel along the straight tracker line)                        */
/* ---------------------------------------------------------------------- */

static double o_face_dist(double pos, double o, double d)
{
    double r = (pos - o) / d;
    double f = r - floor(r);
    double m = f < 1.0 - f ? f : 1.0 - f;
    return m * d;
}

/* Straight line p(s) = T + s D, s in [0, S], D in lab mm per mm of depth.
 * On a hit returns 1 and *s_hit = parameter where the line first enters a
 * voxel whose mask byte is nonzero.  *margin (if not NULL) is lowered to the
 * smallest distance (mm) between a crossing point and a face of another axis.
 * *cond (if not NULL) is raised to the conditioning of the crossing into the
 * hit voxel: the line's length per unit of travel across the crossed face,
 * |D| / |D_a| (1 when the line starts inside that voxel) -- how far a
 * position error moves that crossing along the line. */
int o_hull_entry(const o_cfg *g, const uint8_t *mask, const double T[3], const double D[3],
                 double S, double *s_hit, double *margin, double *cond)
{
    const int32_t n[3] = {g->nx, g->ny, g->nz};
    const double d[3] = {g->dx, g->dy, g->dz};
    const double o[3] = {g->ox, g->oy, g->oz};
    double s_lo = 0.0, s_hi = S;
    int cross_axis = -1; /* axis of the face crossed into the current voxel */
    for (int a = 0; a < 3; ++a) {
        double lo = o[a], hi = o[a] + n[a] * d[a];
        if (D[a] == 0.0) {
            if (T[a] < lo || T[a] >= hi) return 0;
        } else {
            double s1 = (lo - T[a]) / D[a], s2 = (hi - T[a]) / D[a];
            if (s1 > s2) { double tmp = s1; s1 = s2; s2 = tmp; }
            if (s1 > s_lo) { s_lo = s1; cross_axis = a; }
            if (s2 < s_hi) s_hi = s2;
        }
    }
    const double dlen = sqrt(D[0] * D[0] + D[1] * D[1] + D[2] * D[2]);
    if (!(s_lo < s_hi)) return 0;
    int32_t iv[3];
    for (int a = 0; a < 3; ++a) {
        double r = (T[a] + s_lo * D[a] - o[a]) / d[a];
        double fl = floor(r);
        int32_t k = (int32_t)fl;
        if (r == fl && D[a] < 0.0) k -= 1; /* on a face: the voxel we move into */
        if (k < 0) k = 0;
        if (k > n[a] - 1) k = n[a] - 1;
        iv[a] = k;
    }
    double s_cur = s_lo;
    for (;;) {
        int64_t j = iv[0] + (int64_t)n[0] * (iv[1] + (int64_t)n[1] * iv[2]);
        if (mask == NULL || mask[j]) {
            *s_hit = s_cur;
            if (cond && cross_axis >= 0) {
                double c = dlen / fabs(D[cross_axis]);
                if (c > *cond) *cond = c;
            }
            return 1;
        }
        double tm[3];
        double s_next = INFINITY;
        for (int a = 0; a < 3; ++a) {
            if (D[a] > 0.0)
                tm[a] = (o[a] + (iv[a] + 1) * d[a] - T[a]) / D[a];
            else if (D[a] < 0.0)
                tm[a] = (o[a] + iv[a] * d[a] - T[a]) / D[a];
            else
                tm[a] = INFINITY;
            if (tm[a] < s_next) s_next = tm[a];
        }
        if (!(s_next < s_hi)) return 0;
        for (int a = 0; a < 3; ++a) {
            if (tm[a] == s_next) {
                iv[a] += D[a] > 0.0 ? 1 : -1;
                if (cross_axis < 0 || fabs(D[a]) < fabs(D[cross_axis]) || tm[cross_axis] != s_next)
                    cross_axis = a;
            } else if (margin) {
                double m = o_face_dist(T[a] + s_next * D[a], o[a], d[a]);
                if (m < *margin) *margin = m;
            }
        }
        s_cur = s_next;
        for (int a = 0; a < 3; ++a)
            if (iv[a] < 0 || iv[a] >= n[a]) return 0;
    }
}

/* Per-proton hull-frame state.  Beam frame of gantry angle phi:
 * u = (cos phi, sin phi, 0), t = (-sin phi, cos phi, 0), v = z.
 * h[0..11] = in_x, in_y, in_z, out_x, out_y, out_z, theta_in, psi_in,
 *            theta_out, psi_out, phi, wepl.
 * st[0..11] = u_in, u_out, t0, th0, v0, ps0, t2, th2, v2, ps2, cos phi, sin phi. */
static int o_state_one(const o_cfg *g, const uint8_t *mask, const double *const h[12], int64_t i,
                       double st[12], double *margin, double *cond)
{
    double c = cos(h[10][i]), s = sin(h[10][i]);
    double ua = h[0][i] * c + h[1][i] * s, ta = -h[0][i] * s + h[1][i] * c, va = h[2][i];
    double ub = h[3][i] * c + h[4][i] * s, tb = -h[3][i] * s + h[4][i] * c, vb = h[5][i];
    double tti = tan(h[6][i]), tpi = tan(h[7][i]), tto = tan(h[8][i]), tpo = tan(h[9][i]);
    memset(st, 0, 12 * sizeof(double));
    st[10] = c;
    st[11] = s;
    if (!(ub > ua)) return 0;
    double S = ub - ua;
    double Ti[3] = {h[0][i], h[1][i], h[2][i]};
    double Di[3] = {c - tti * s, s + tti * c, tpi};
    double To[3] = {h[3][i], h[4][i], h[5][i]};
    double Do[3] = {-(c - tto * s), -(s + tto * c), -tpo};
    double s_in, s_out;
    if (!o_hull_entry(g, mask, Ti, Di, S, &s_in, margin, cond)) return 0;
    if (!o_hull_entry(g, mask, To, Do, S, &s_out, margin, cond)) return 0;
    double u_in = ua + s_in, u_out = ub - s_out;
    if (!(u_out > u_in)) return 0;
    st[0] = u_in;
    st[1] = u_out;
    st[2] = ta + tti * s_in;
    st[3] = h[6][i];
    st[4] = va + tpi * s_in;
    st[5] = h[7][i];
    st[6] = tb - tto * s_out;
    st[7] = h[8][i];
    st[8] = vb - tpo * s_out;
    st[9] = h[9][i];
    return 1;
}

int o_prepare(const o_cfg *g, const uint8_t *mask, int64_t n, const double *const h[12],
              double *states, int32_t *valid, double *margin)
{
#pragma omp parallel for schedule(dynamic, 256)
    for (int64_t i = 0; i < n; ++i) {
        double m = INFINITY;
        valid[i] = o_state_one(g, mask, h, i, states + 12 * i, &m, NULL);
        if (margin) margin[i] = m;
    }
    return 0;
}

/* ---------------------------------------------------------------------- */
/* MLP polyline                                                             */
/* ---------------------------------------------------------------------- */

/* Number of interior samples: depths k*du (k >= 1) with k*du < L - dend. */
static int64_t o_n_interior(const o_cfg *g, double L)
{
    double lim = L - g->dend;
    int64_t k = 0;
    while ((double)(k + 1) * g->du < lim) ++k;
    return k;
}

/* Lab points (mm) of the MLP polyline: the hull entry point, the interior
 * samples, the hull exit point.  Returns the number of points (0 if the
 * proton misses the hull); writes at most cap points. */
static int64_t o_polyline(const o_cfg *g, const double st[12], int ok, double *pts, int64_t cap,
                          double *margin)
{
    if (!ok) return 0;
    double c = st[10], s = st[11];
    double u_in = st[0], L = st[1] - st[0];
    double t0 = st[2], th0 = st[3], v0 = st[4], ps0 = st[5];
    double t2 = st[6], th2 = st[7], v2 = st[8], ps2 = st[9];
    int64_t K = o_n_interior(g, L);
    if (margin) {
        double lim = L - g->dend;
        double m1 = lim - K * g->du, m2 = (K + 1) * g->du - lim;
        if (m1 < *margin) *margin = m1;
        if (m2 < *margin) *margin = m2;
    }
    int64_t np = 0;
#define O_PUT(U, T, V)                                   \
    do {                                                 \
        if (np < cap) {                                  \
            pts[3 * np + 0] = (U) * c - (T) * s;         \
            pts[3 * np + 1] = (U) * s + (T) * c;         \
            pts[3 * np + 2] = (V);                       \
        }                                                \
        ++np;                                            \
    } while (0)
    O_PUT(u_in, t0, v0);
    /* MLP in coordinates relative to the entry point (the MLP is linear in
     * (y0, y2) and commutes with a common shift of both positions). */
    double yt0[2] = {0.0, th0}, yt2[2] = {(t2 - t0) / 10.0, th2};
    double yv0[2] = {0.0, ps0}, yv2[2] = {(v2 - v0) / 10.0, ps2};
    for (int64_t k = 1; k <= K; ++k) {
        double w = k * g->du;
        double yt1[2], yv1[2];
        o_mlp_point(g, yt0, yt2, L / 10.0, w / 10.0, yt1);
        o_mlp_point(g, yv0, yv2, L / 10.0, w / 10.0, yv1);
        O_PUT(u_in + w, t0 + 10.0 * yt1[0], v0 + 10.0 * yv1[0]);
    }
    O_PUT(st[1], t2, v2);
#undef O_PUT
    return np;
}

int o_mlp_points(const o_cfg *g, const uint8_t *mask, int64_t n, const double *const h[12],
                 int32_t max_pts, double *pts, int32_t *npts)
{
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t i = 0; i < n; ++i) {
        double st[12];
        int ok = o_state_one(g, mask, h, i, st, NULL, NULL);
        npts[i] = (int32_t)o_polyline(g, st, ok, pts + (int64_t)3 * max_pts * i, max_pts, NULL);
    }
    return 0;
}

/* ---------------------------------------------------------------------- */
/* Voxel walk (3D Amanatides-Woo along each polyline segment)              */
/* ---------------------------------------------------------------------- */

/* The walk produces "visits": maximal runs of the path inside one voxel.
 * Visits in voxels outside the grid or outside the hull are dropped
 * afterwards; a row is the remaining visits in path order. */
typedef struct {
    const o_cfg *g;
    const uint8_t *mask;
    int32_t *out_j;
    double *out_l;
    int64_t cap, n;
    int32_t cur[3];
    double cur_len;
    int have;
} o_row;

static void o_row_flush(o_row *r)
{
    if (!r->have) return;
    r->have = 0;
    const o_cfg *g = r->g;
    if (r->cur[0] < 0 || r->cur[0] >= g->nx || r->cur[1] < 0 || r->cur[1] >= g->ny ||
        r->cur[2] < 0 || r->cur[2] >= g->nz)
        return;
    int64_t j = r->cur[0] + (int64_t)g->nx * (r->cur[1] + (int64_t)g->ny * r->cur[2]);
    if (r->mask && !r->mask[j]) return;
    if (r->n < r->cap) {
        r->out_j[r->n] = (int32_t)j;
        r->out_l[r->n] = r->cur_len;
    }
    r->n++;
}

static void o_row_add(o_row *r, const int32_t iv[3], double len)
{
    if (!(len > 0.0)) return;
    if (r->have && r->cur[0] == iv[0] && r->cur[1] == iv[1] && r->cur[2] == iv[2]) {
        r->cur_len += len;
        return;
    }
    o_row_flush(r);
    r->have = 1;
    r->cur[0] = iv[0];
    r->cur[1] = iv[1];
    r->cur[2] = iv[2];
    r->cur_len = len;
}

/* Walk the polyline pts[0..np-1] (lab mm).  Per segment: the start voxel is
 * floor of the start point, a start point exactly on a face belonging to the
 * voxel the segment moves into; equal crossing parameters on several axes
 * step all of them at once (no zero-length chord).  Returns the row length. */
static int64_t o_walk_row(const o_cfg *g, const uint8_t *mask, const double *pts, int64_t np,
                          int32_t *out_j, double *out_l, int64_t cap, double *margin, double *cond)
{
    const double d[3] = {g->dx, g->dy, g->dz};
    const double o[3] = {g->ox, g->oy, g->oz};
    o_row r;
    memset(&r, 0, sizeof r);
    r.g = g;
    r.mask = mask;
    r.out_j = out_j;
    r.out_l = out_l;
    r.cap = cap;
    double prevD[3] = {0.0, 0.0, 0.0};
    for (int64_t k = 0; k + 1 < np; ++k) {
        const double *A = pts + 3 * k, *B = pts + 3 * k + 3;
        double gA[3], D[3], len2 = 0.0;
        for (int a = 0; a < 3; ++a) {
            /* both vertices in grid units by the same expression, so that a
             * segment ends exactly where the next one starts */
            gA[a] = (A[a] - o[a]) / d[a];
            D[a] = (B[a] - o[a]) / d[a] - gA[a];
            len2 += (B[a] - A[a]) * (B[a] - A[a]);
        }
        double len = sqrt(len2);
        if (margin && k > 0) {
            /* a vertex where the path turns back along an axis can graze a face */
            for (int a = 0; a < 3; ++a)
                if (prevD[a] * D[a] <= 0.0) {
                    double m = o_face_dist(A[a], o[a], d[a]);
                    if (m < *margin) *margin = m;
                }
        }
        memcpy(prevD, D, sizeof D);
        if (!(len > 0.0)) continue;
        int32_t iv[3];
        double tm[3], td[3];
        for (int a = 0; a < 3; ++a) {
            double fl = floor(gA[a]);
            iv[a] = (int32_t)fl;
            if (gA[a] == fl && D[a] < 0.0) iv[a] -= 1;
            if (D[a] > 0.0) {
                tm[a] = (iv[a] + 1 - gA[a]) / D[a];
                td[a] = 1.0 / D[a];
            } else if (D[a] < 0.0) {
                tm[a] = (iv[a] - gA[a]) / D[a];
                td[a] = -1.0 / D[a];
            } else {
                tm[a] = INFINITY;
                td[a] = INFINITY;
            }
        }
        double t = 0.0;
        for (;;) {
            double tn = tm[0];
            if (tm[1] < tn) tn = tm[1];
            if (tm[2] < tn) tn = tm[2];
            if (tn >= 1.0) {
                o_row_add(&r, iv, (1.0 - t) * len);
                break;
            }
            o_row_add(&r, iv, (tn - t) * len);
            int stepped = 0;
            for (int a = 0; a < 3; ++a)
                if (tm[a] == tn) ++stepped;
            for (int a = 0; a < 3; ++a) {
                if (tm[a] == tn) {
                    iv[a] += D[a] > 0.0 ? 1 : -1;
                    tm[a] += td[a];
                    /* path length per unit of travel across the crossed face:
                     * how far a sideways error moves this crossing */
                    if (cond) {
                        double c = len / fabs(D[a] * d[a]);
                        if (c > *cond) *cond = c;
                    }
                } else if (margin) {
                    double m = o_face_dist(A[a] + tn * D[a] * d[a], o[a], d[a]);
                    if (m < *margin) *margin = m;
                }
            }
            if (stepped > 1 && margin) *margin = 0.0;
            t = tn;
        }
    }
    o_row_flush(&r);
    return r.n;
}

/* Rows of A in path order.  Two passes: with out_j == NULL only the row
 * lengths are written to rowptr[1..n] (rowptr[0] = 0 is left to the caller's
 * prefix sum); otherwise rowptr must hold the offsets. */
int o_rows(const o_cfg *g, const uint8_t *mask, int64_t n, const double *const h[12],
           int64_t *rowptr, int32_t *out_j, double *out_l, double *margin, double *cond)
{
    int err = 0;
#pragma omp parallel
    {
        int64_t cap_pts = 1024;
        double *pts = (double *)malloc(sizeof(double) * 3 * cap_pts);
#pragma omp for schedule(dynamic, 64)
        for (int64_t i = 0; i < n; ++i) {
            double st[12];
            double m = INFINITY, cd = 1.0;
            int ok = o_state_one(g, mask, h, i, st, &m, &cd);
            int64_t np = o_polyline(g, st, ok, pts, cap_pts, &m);
            if (np > cap_pts) {
                cap_pts = np;
                pts = (double *)realloc(pts, sizeof(double) * 3 * cap_pts);
                m = INFINITY;
                cd = 1.0;
                o_state_one(g, mask, h, i, st, &m, &cd);
                np = o_polyline(g, st, ok, pts, cap_pts, &m);
            }
            if (out_j == NULL) {
                rowptr[i + 1] = o_walk_row(g, mask, pts, np, NULL, NULL, 0, &m, &cd);
            } else {
                int64_t cap = rowptr[i + 1] - rowptr[i];
                int64_t got = o_walk_row(g, mask, pts, np, out_j + rowptr[i], out_l + rowptr[i],
                                         cap, &m, &cd);
                if (got != cap) {
#pragma omp atomic write
                    err = 1;
                }
            }
            if (margin) margin[i] = m;
            if (cond) cond[i] = cd;
        }
        free(pts);
    }
    return err ? -1 : 0;
}

/* Walk one caller-given polyline (lab mm); used by the brute-force pins. */
int64_t o_walk(const o_cfg *g, const uint8_t *mask, int64_t np, const double *pts, int32_t *out_j,
               double *out_l, int64_t cap, double *margin)
{
    return o_walk_row(g, mask, pts, np, out_j, out_l, cap, margin, NULL);
}

/* ---------------------------------------------------------------------- */
/* DROP (Sec. IV-B; Penfold, Schulte, Censor et al. 2010)                   */
/* ---------------------------------------------------------------------- */

/* CSR rows with one entry per (i, j) (duplicates already summed) and all
 * stored values > 0.  x is updated in place. */
int o_drop(int64_t n_vox, int64_t m, const int64_t *rowptr, const int32_t *idx, const double *len,
           const double *b, int32_t iters, double lambda, int64_t block, double *x)
{
    if (block < 1) return -1;
    double *num = (double *)calloc((size_t)n_vox, sizeof(double));
    int64_t *cnt = (int64_t *)calloc((size_t)n_vox, sizeof(int64_t));
    double *r = (double *)malloc(sizeof(double) * (size_t)(block > m ? (m > 0 ? m : 1) : block));
    if (!num || !cnt || !r) {
        free(num);
        free(cnt);
        free(r);
        return -2;
    }
    for (int32_t it = 0; it < iters; ++it) {
        for (int64_t t0 = 0; t0 < m; t0 += block) {
            int64_t t1 = t0 + block < m ? t0 + block : m;
            /* residual of every row of the block against the frozen x */
#pragma omp parallel for schedule(static)
            for (int64_t i = t0; i < t1; ++i) {
                double s = 0.0, q = 0.0;
                for (int64_t e = rowptr[i]; e < rowptr[i + 1]; ++e) {
                    s += len[e] * x[idx[e]];
                    q += len[e] * len[e];
                }
                r[i - t0] = q > 0.0 ? (b[i] - s) / q : 0.0;
            }
            /* sum_i a_ij r_i and s_j over the block */
            for (int64_t i = t0; i < t1; ++i)
                for (int64_t e = rowptr[i]; e < rowptr[i + 1]; ++e) {
                    num[idx[e]] += len[e] * r[i - t0];
                    cnt[idx[e]] += 1;
                }
            /* x_j += lambda * num_j / s_j on the voxels the block touched */
            for (int64_t i = t0; i < t1; ++i)
                for (int64_t e = rowptr[i]; e < rowptr[i + 1]; ++e) {
                    int32_t j = idx[e];
                    if (cnt[j] > 0) {
                        x[j] += lambda * num[j] / (double)cnt[j];
                        num[j] = 0.0;
                        cnt[j] = 0;
                    }
                }
        }
    }
    free(num);
    free(cnt);
    free(r);
    return 0;
}

int o_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
