"""Pins of the FP64 oracle against things other than itself.

Each test ties one oracle function to a closed form, an independent numerical
method, a brute-force computation or a textbook special case, chosen so that
a plausible slip (a dropped term, a wrong sign or weight, a transposed matrix,
a wrong tie rule) fails at least one of them.  CPU only.
"""
import math

import numpy as np
import pytest
import scipy.integrate as si
import scipy.sparse as sp

import oracle as O
import synth

pytestmark = pytest.mark.filterwarnings("ignore::DeprecationWarning")

X0 = 36.08
E0 = 13.6


def _geo(shape=(16, 16, 16), voxel=(1.0, 1.0, 1.0), origin=None, mask=None, **kw):
    if origin is None:
        origin = tuple(-0.5 * n * d for n, d in zip(shape, voxel))
    return O.Geometry(shape, voxel, origin, mask=mask, **kw)


# --------------------------------------------------------------------------
# Scattering matrices (MLP prior of Schulte et al. 2008, cited in Sec. I)
# --------------------------------------------------------------------------

def test_gauss_legendre_rule_matches_numpy():
    # the oracle's 5-point rule, recovered by integrating monomials exactly
    geo = _geo(coef=(1.0, 0, 0, 0, 0, 0), highland=False)
    x, w = np.polynomial.legendre.leggauss(5)
    assert np.isclose(w.sum(), 2.0)
    # int_0^h (h-u)^2 du = h^3/3, (h-u) -> h^2/2, 1 -> h; prefactor E0^2/X0
    for h in (0.1, 1.0, 7.3):
        S = O.sigma(geo, 0.0, h)
        pre = E0 * E0 / X0
        assert np.allclose(S, pre * np.array([h ** 3 / 3, h ** 2 / 2, h]), rtol=1e-13)


@pytest.mark.parametrize("ua,ub", [(0.0, 0.1), (0.0, 12.0), (3.0, 17.5), (19.99, 20.0), (0.0, 28.0)])
def test_sigma_matches_adaptive_quadrature(ua, ub):
    geo = _geo()
    f = np.polynomial.Polynomial(O.COEF_200MEV_WATER)
    pre = E0 ** 2 * (1 + 0.038 * math.log((ub - ua) / X0)) ** 2 / X0
    want = [si.quad(lambda u, n=n: (ub - u) ** n * f(u), ua, ub, epsabs=0, epsrel=1e-13)[0]
            for n in (2, 1, 0)]
    got = O.sigma(geo, ua, ub)
    assert np.allclose(got, pre * np.array(want), rtol=1e-11, atol=0)


def test_sigma_is_positive_definite_over_torso_depths():
    geo = _geo()
    for L in np.linspace(0.05, 30.0, 40):
        s = O.sigma(geo, 0.0, L)
        assert s[0] > 0 and s[2] > 0 and s[0] * s[2] - s[1] ** 2 > 0


# --------------------------------------------------------------------------
# MLP state
# --------------------------------------------------------------------------

def _R(d):
    return np.array([[1.0, d], [0.0, 1.0]])


@pytest.mark.parametrize("L", [4.4, 17.7, 26.0])
def test_mlp_straight_line_invariant(L):
    # exit state on the straight continuation of the entry state => straight path
    geo = _geo()
    y0 = np.array([0.37, 0.004])
    y2 = _R(L) @ y0
    for u1 in np.linspace(0.1, L - 0.1, 9):
        y1 = O.mlp_point(geo, y0, y2, L, u1)
        assert np.allclose(y1, _R(u1) @ y0, rtol=0, atol=1e-12)


def test_mlp_zero_angle_zero_offset_is_on_axis():
    geo = _geo()
    for u1 in (0.5, 5.0, 9.5):
        assert np.allclose(O.mlp_point(geo, [0.0, 0.0], [0.0, 0.0], 10.0, u1), 0.0, atol=1e-15)


@pytest.mark.parametrize("L", [2.0, 15.0])
def test_mlp_uniform_scattering_is_cubic_hermite(L):
    # constant 1/(beta^2 p^2), no log term: the conditional mean of an
    # integrated Brownian angle given both end states is the cubic Hermite
    # interpolant of (t0, theta0) and (t2, theta2)
    geo = _geo(coef=(3e-5, 0, 0, 0, 0, 0), highland=False)
    t0, th0, t2, th2 = 0.2, 0.01, -0.15, -0.02
    for u in np.linspace(0.05 * L, 0.95 * L, 11):
        s = u / L
        h00, h10 = 2 * s ** 3 - 3 * s ** 2 + 1, s ** 3 - 2 * s ** 2 + s
        h01, h11 = -2 * s ** 3 + 3 * s ** 2, s ** 3 - s ** 2
        t = h00 * t0 + h10 * L * th0 + h01 * t2 + h11 * L * th2
        dh00, dh10 = (6 * s ** 2 - 6 * s) / L, (3 * s ** 2 - 4 * s + 1) / L
        dh01, dh11 = (-6 * s ** 2 + 6 * s) / L, (3 * s ** 2 - 2 * s) / L
        th = dh00 * t0 + dh10 * L * th0 + dh01 * t2 + dh11 * L * th2
        y1 = O.mlp_point(geo, [t0, th0], [t2, th2], L, u)
        assert np.allclose(y1, [t, th], rtol=0, atol=1e-10)


def test_mlp_equals_gaussian_conditional_mean():
    # textbook Gaussian conditioning: y1 ~ N(R0 y0, S1), y2 | y1 ~ N(R1 y1, S2)
    geo = _geo()
    rng = np.random.default_rng(7)
    for _ in range(20):
        L = rng.uniform(2.0, 27.0)
        u1 = rng.uniform(0.05, L - 0.05)
        y0 = np.array([rng.normal(0, 1.0), rng.normal(0, 0.01)])
        y2 = np.array([rng.normal(0, 1.0), rng.normal(0, 0.03)])
        a = O.sigma(geo, 0.0, u1)
        b = O.sigma(geo, u1, L)
        S1 = np.array([[a[0], a[1]], [a[1], a[2]]])
        S2 = np.array([[b[0], b[1]], [b[1], b[2]]])
        R0, R1 = _R(u1), _R(L - u1)
        cov12 = S1 @ R1.T
        cov22 = R1 @ S1 @ R1.T + S2
        want = R0 @ y0 + cov12 @ np.linalg.solve(cov22, y2 - R1 @ R0 @ y0)
        got = O.mlp_point(geo, y0, y2, L, u1)
        assert np.allclose(got, want, rtol=1e-9, atol=1e-12)


def test_mlp_endpoint_limits_and_mirror():
    geo = _geo()
    y0, y2, L = np.array([0.3, 0.01]), np.array([-0.2, -0.03]), 12.0
    near0 = O.mlp_point(geo, y0, y2, L, 1e-4)
    nearL = O.mlp_point(geo, y0, y2, L, L - 1e-4)
    assert abs(near0[0] - y0[0]) < 1e-5 and abs(nearL[0] - y2[0]) < 1e-5
    m = O.mlp_point(geo, -y0, -y2, L, 5.0)
    assert np.allclose(m, -O.mlp_point(geo, y0, y2, L, 5.0), atol=1e-15)


# --------------------------------------------------------------------------
# Hull entry along a straight line
# --------------------------------------------------------------------------

def _ball_mask(shape, r):
    nx, ny, nz = shape
    z, y, x = np.meshgrid(np.arange(nz) + 0.5 - nz / 2, np.arange(ny) + 0.5 - ny / 2,
                          np.arange(nx) + 0.5 - nx / 2, indexing="ij")
    return (x * x + y * y + z * z <= r * r).astype(np.uint8).reshape(-1)


def _slab(T, D, lo, hi):
    s0, s1 = -np.inf, np.inf
    for a in range(3):
        if D[a] == 0:
            if not (lo[a] <= T[a] <= hi[a]):
                return np.inf, -np.inf
        else:
            p, q = (lo[a] - T[a]) / D[a], (hi[a] - T[a]) / D[a]
            s0, s1 = max(s0, min(p, q)), min(s1, max(p, q))
    return s0, s1


def test_hull_entry_matches_brute_force_box_clipping():
    shape = (12, 10, 8)
    mask = _ball_mask(shape, 4.3)
    geo = _geo(shape=shape, mask=mask)
    o = np.array(geo.origin)
    rng = np.random.default_rng(3)
    hull = np.flatnonzero(mask)
    checked = 0
    for _ in range(300):
        T = np.array([-9.0, rng.uniform(-6, 6), rng.uniform(-5, 5)])
        D = np.array([1.0, rng.normal(0, 0.4), rng.normal(0, 0.4)])
        S = 18.0
        best = np.inf
        for j in hull:
            ix, iy, iz = j % shape[0], (j // shape[0]) % shape[1], j // (shape[0] * shape[1])
            lo = o + np.array([ix, iy, iz], dtype=float)
            s0, s1 = _slab(T, D, lo, lo + 1.0)
            s0, s1 = max(s0, 0.0), min(s1, S)
            if s1 > s0:
                best = min(best, s0)
        hit, s, _ = O.hull_entry(geo, T, D, S)
        assert hit == np.isfinite(best)
        if hit:
            assert abs(s - best) < 1e-9
            checked += 1
    assert checked > 50


# --------------------------------------------------------------------------
# Voxel walk
# --------------------------------------------------------------------------

def _brute_row(geo, pts):
    """Chord of each segment in each voxel box by slab clipping, summed per voxel."""
    nx, ny, nz = geo.shape
    o = np.array(geo.origin)
    d = np.array(geo.voxel)
    acc = np.zeros(nx * ny * nz)
    for A, B in zip(pts[:-1], pts[1:]):
        D = B - A
        seg = np.linalg.norm(D)
        for iz in range(nz):
            for iy in range(ny):
                for ix in range(nx):
                    lo = o + d * np.array([ix, iy, iz])
                    s0, s1 = _slab(A, D, lo, lo + d)
                    s0, s1 = max(s0, 0.0), min(s1, 1.0)
                    if s1 > s0:
                        acc[ix + nx * (iy + ny * iz)] += (s1 - s0) * seg
    return acc


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_walk_matches_brute_force_slab_clipping(seed):
    rng = np.random.default_rng(seed)
    geo = _geo(shape=(9, 8, 7), voxel=(1.0, 1.3, 0.8))
    lo = np.array(geo.origin) + 0.01
    hi = -lo
    pts = [rng.uniform(lo, hi)]
    for _ in range(6):
        nxt = pts[-1] + rng.normal(0, 1.5, 3)
        pts.append(np.clip(nxt, lo, hi))
    pts = np.array(pts)
    j, ln, _ = O.walk(geo, pts)
    got = np.bincount(j, weights=ln, minlength=geo.n_vox)
    want = _brute_row(geo, pts)
    assert np.allclose(got, want, atol=1e-9)
    assert abs(ln.sum() - np.linalg.norm(np.diff(pts, axis=0), axis=1).sum()) < 1e-9


def test_walk_axis_aligned_face_to_face_gives_unit_chords():
    geo = _geo(shape=(10, 4, 4), origin=(0.0, 0.0, 0.0))
    fwd = np.array([[0.0, 1.5, 2.5], [10.0, 1.5, 2.5]])
    j, ln, _ = O.walk(geo, fwd)
    assert np.array_equal(j, np.arange(10) + 10 * (1 + 4 * 2))
    assert np.allclose(ln, 1.0, rtol=0, atol=1e-12)
    jb, lb, _ = O.walk(geo, fwd[::-1])   # start exactly on the far face moving -x
    assert np.array_equal(jb, j[::-1]) and np.allclose(lb, 1.0, rtol=0, atol=1e-12)


def test_walk_merges_segments_inside_one_voxel_and_keeps_path_order():
    geo = _geo(shape=(6, 6, 6), origin=(0.0, 0.0, 0.0))
    pts = np.array([[0.1, 0.2, 0.3], [0.3, 0.4, 0.3], [0.6, 0.5, 0.4], [0.9, 0.9, 0.8]])
    j, ln, _ = O.walk(geo, pts)
    assert j.tolist() == [0]
    assert np.isclose(ln[0], np.linalg.norm(np.diff(pts, axis=0), axis=1).sum())
    # a diagonal line: consecutive visits are 26-neighbours, in path order
    line = np.array([[0.2, 0.1, 0.05], [5.7, 5.9, 4.1]])
    j, ln, _ = O.walk(geo, line)
    ijk = np.stack([j % 6, (j // 6) % 6, j // 36], axis=1)
    assert np.all(np.abs(np.diff(ijk, axis=0)) <= 1)
    assert np.all(np.diff(ijk, axis=0).sum(axis=1) > 0)


def test_walk_drops_voxels_outside_hull_and_grid():
    mask = np.zeros(6 * 6 * 6, dtype=np.uint8)
    mask[[1, 2]] = 1                                  # voxels (1,0,0) and (2,0,0)
    geo = _geo(shape=(6, 6, 6), origin=(0.0, 0.0, 0.0), mask=mask)
    line = np.array([[-3.0, 0.5, 0.5], [9.0, 0.5, 0.5]])
    j, ln, _ = O.walk(geo, line)
    assert j.tolist() == [1, 2] and np.allclose(ln, 1.0)


# --------------------------------------------------------------------------
# Proton pipeline: hull states, MLP polyline and rows
# --------------------------------------------------------------------------

def _one_proton(phi, t, v, th_in=0.0, ps_in=0.0, th_out=0.0, ps_out=0.0, U=60.0, dt=0.0, dv=0.0):
    c, s = math.cos(phi), math.sin(phi)
    lab = lambda u, tt, vv: (u * c - tt * s, u * s + tt * c, vv)
    a = lab(-U, t, v)
    b = lab(U, t + dt, v + dv)
    return {"in_x": [a[0]], "in_y": [a[1]], "in_z": [a[2]], "out_x": [b[0]], "out_y": [b[1]],
            "out_z": [b[2]], "theta_in": [th_in], "psi_in": [ps_in], "theta_out": [th_out],
            "psi_out": [ps_out], "phi": [phi], "wepl": [10.0]}


def test_zero_angle_proton_through_uniform_phantom_is_straight():
    shape = (40, 40, 8)
    geo = _geo(shape=shape, mask=None)
    for phi in (0.3, 1.1, 2.6):
        h = _one_proton(phi, t=3.217, v=0.41)
        st, ok, _ = O.prepare(geo, h)
        assert ok[0]
        pts, npts = O.mlp_points(geo, h, 200)
        p = pts[0, :npts[0]]
        c, s = math.cos(phi), math.sin(phi)
        tt = -p[:, 0] * s + p[:, 1] * c
        assert np.allclose(tt, 3.217, atol=1e-9) and np.allclose(p[:, 2], 0.41, atol=1e-12)
        rp, j, ln, _ = O.rows(geo, h)
        L = st[0, 1] - st[0, 0]
        assert abs(ln.sum() - L) < 1e-9


def test_prepare_states_lie_on_the_tracker_lines():
    mask = _ball_mask((30, 30, 10), 9.0)
    geo = _geo(shape=(30, 30, 10), mask=mask)
    h = _one_proton(0.7, t=2.0, v=0.5, th_in=0.02, ps_in=-0.01, th_out=-0.03, ps_out=0.015,
                    dt=1.0, dv=-0.4)
    st, ok, _ = O.prepare(geo, h)
    assert ok[0]
    u_in, u_out, t0, th0, v0, ps0, t2, th2, v2, ps2, c, s = st[0]
    assert np.isclose(t0, 2.0 + math.tan(0.02) * (u_in + 60.0))
    assert np.isclose(v0, 0.5 + math.tan(-0.01) * (u_in + 60.0))
    assert np.isclose(t2, 3.0 + math.tan(-0.03) * (u_out - 60.0))
    assert np.isclose(v2, 0.1 + math.tan(0.015) * (u_out - 60.0))
    assert -9.5 < u_in < -7.0 and 7.0 < u_out < 9.5
    # the entry point sits on a face of a hull voxel
    x = u_in * c - t0 * s
    y = u_in * s + t0 * c
    r = np.array([x, y, v0]) - np.array(geo.origin)
    assert np.min(np.abs(r - np.round(r))) < 1e-9


def test_mlp_polyline_starts_and_ends_at_the_hull_states():
    # the MLP reproduces the measured (hull-projected) entry and exit points:
    # the first and last vertices of the polyline are those points
    mask = _ball_mask((30, 30, 10), 9.0)
    geo = _geo(shape=(30, 30, 10), mask=mask)
    for phi, th_in, th_out in ((0.7, 0.02, -0.03), (2.2, -0.015, 0.01), (4.0, 0.0, 0.025)):
        h = _one_proton(phi, t=1.5, v=-0.3, th_in=th_in, ps_in=0.01, th_out=th_out, ps_out=-0.02,
                        dt=0.8, dv=0.3)
        st, ok, _ = O.prepare(geo, h)
        assert ok[0]
        u_in, u_out, t0, th0, v0, ps0, t2, th2, v2, ps2, c, s = st[0]
        pts, npts = O.mlp_points(geo, h, 200)
        p = pts[0, :npts[0]]
        entry = np.array([u_in * c - t0 * s, u_in * s + t0 * c, v0])
        exit_ = np.array([u_out * c - t2 * s, u_out * s + t2 * c, v2])
        assert np.allclose(p[0], entry, rtol=0, atol=1e-12)
        assert np.allclose(p[-1], exit_, rtol=0, atol=1e-12)
        assert npts[0] > 3 and np.all(np.isfinite(p))


def _beam_proton(phi, ua, ta, va, ub, tb, vb, th_in, ps_in, th_out, ps_out):
    """One history given by its tracker points in the beam frame of phi (mm)."""
    c, s = math.cos(phi), math.sin(phi)
    return {"in_x": [ua * c - ta * s], "in_y": [ua * s + ta * c], "in_z": [va],
            "out_x": [ub * c - tb * s], "out_y": [ub * s + tb * c], "out_z": [vb],
            "theta_in": [th_in], "psi_in": [ps_in], "theta_out": [th_out], "psi_out": [ps_out],
            "phi": [phi], "wepl": [10.0]}


def _beam_coords(p, phi):
    c, s = math.cos(phi), math.sin(phi)
    return p[:, 0] * c + p[:, 1] * s, -p[:, 0] * s + p[:, 1] * c, p[:, 2]


def _interior_count(L, du, dend):
    # brute force over candidate sample indices: k >= 1 with k du < L - dend
    return sum(1 for k in range(1, 100000) if k * du < L - dend)


@pytest.mark.parametrize("du", [1.0, 0.7])
def test_polyline_interior_straight_line_with_angles_and_offsets(du):
    # Tracker points strictly inside the grid box with every voxel in the hull:
    # the hull entry and exit are the tracker points themselves.  An exit state
    # on the straight continuation of the entry state (theta, psi != 0, offsets
    # != 0, gantry angle != 0) must give a polyline whose interior vertices lie
    # on that line, at beam depths u_in + k du exactly.  A unit slip between mm
    # and cm in the sample depth, the path depth or the exit offset bends it.
    geo = _geo(shape=(60, 60, 20), du=du)
    th, ps = 0.031, -0.017
    ua, ta, va, L = -22.3, 4.1, -2.7, 41.37
    for phi in (0.0, 0.9, 2.4, 5.1):
        h = _beam_proton(phi, ua, ta, va, ua + L, ta + th * L, va + ps * L, th, ps, th, ps)
        st, ok, _ = O.prepare(geo, h)
        assert ok[0] and abs(st[0, 0] - ua) < 1e-12 and abs(st[0, 1] - (ua + L)) < 1e-12
        pts, npts = O.mlp_points(geo, h, 200)
        K = _interior_count(L, du, geo.dend)
        assert npts[0] == K + 2
        u, t, v = _beam_coords(pts[0, :npts[0]], phi)
        depths = np.concatenate([[ua], ua + du * np.arange(1, K + 1), [ua + L]])
        assert np.allclose(u, depths, rtol=0, atol=1e-9)
        assert np.allclose(t, ta + th * (u - ua), rtol=0, atol=1e-9)
        assert np.allclose(v, va + ps * (u - ua), rtol=0, atol=1e-9)


@pytest.mark.parametrize("L", [10.0, 10.0 - 1e-6, 10.0 + 5e-4, 10.0 + 2e-3, 0.5, 1.0005, 1.0015])
def test_polyline_sample_count_follows_the_exit_margin(L):
    # interior samples sit at k du (k >= 1) strictly below L - dend: at
    # L = 10 + 5e-4 the 10th sample is within dend of the exit and is left out,
    # at L = 10 + 2e-3 it is kept
    geo = _geo(shape=(40, 40, 10))
    ua = -12.0
    h = _beam_proton(0.4, ua, 1.0, 0.5, ua + L, 1.0, 0.5, 0.0, 0.0, 0.0, 0.0)
    pts, npts = O.mlp_points(geo, h, 64)
    K = _interior_count(L, 1.0, 1e-3)
    assert npts[0] == K + 2
    u, _, _ = _beam_coords(pts[0, :npts[0]], 0.4)
    assert np.allclose(u[1:-1], ua + np.arange(1, K + 1), rtol=0, atol=1e-9)


def _sigma_quad_cm(ua, ub):
    """Scattering matrix of depths [ua, ub] (cm) by adaptive quadrature."""
    f = np.polynomial.Polynomial(O.COEF_200MEV_WATER)
    pre = E0 ** 2 * (1 + 0.038 * math.log((ub - ua) / X0)) ** 2 / X0
    m = [si.quad(lambda u, n=n: (ub - u) ** n * f(u), ua, ub, epsabs=0, epsrel=1e-13)[0]
         for n in (2, 1, 0)]
    return pre * np.array([[m[0], m[1]], [m[1], m[2]]])


def test_polyline_interior_is_the_gaussian_conditional_mean_in_cm():
    # A curved path: each interior vertex (lab mm) must be the conditional mean
    # of the scattering model with depths and positions converted to cm here
    # (the unit of the 1/(beta^2 p^2) fit), conditioned on the hull entry and
    # exit states.  Computed by adaptive quadrature and textbook Gaussian
    # conditioning, independently of the oracle's moments.
    geo = _geo(shape=(80, 80, 24))
    for phi, (ta, th_in, tb, th_out), (va, ps_in, vb, ps_out) in (
            (0.6, (3.0, 0.02, -1.5, -0.035), (1.0, -0.01, 2.2, 0.025)),
            (3.9, (-6.0, -0.04, -2.0, 0.05), (-3.0, 0.03, -4.5, -0.02))):
        ua, ub = -31.0, 33.5
        h = _beam_proton(phi, ua, ta, va, ub, tb, vb, th_in, ps_in, th_out, ps_out)
        pts, npts = O.mlp_points(geo, h, 128)
        u, t, v = _beam_coords(pts[0, :npts[0]], phi)
        Lc = (ub - ua) / 10.0
        worst = 0.0
        for k in range(1, npts[0] - 1):
            w = float(k)                      # mm below the entry (du = 1 mm)
            wc = w / 10.0
            S1, S2 = _sigma_quad_cm(0.0, wc), _sigma_quad_cm(wc, Lc)
            R0, R1 = _R(wc), _R(Lc - wc)
            gain = S1 @ R1.T @ np.linalg.inv(R1 @ S1 @ R1.T + S2)
            for (p0, a0, p2, a2), got in (((ta, th_in, tb, th_out), t[k]), ((va, ps_in, vb, ps_out), v[k])):
                y0 = np.array([p0 / 10.0, a0])
                y2 = np.array([p2 / 10.0, a2])
                y1 = R0 @ y0 + gain @ (y2 - R1 @ R0 @ y0)
                worst = max(worst, abs(10.0 * y1[0] - got))
            assert abs(u[k] - (ua + w)) < 1e-9
        assert worst < 1e-9, worst
        # the path is curved: far from the chord between its end points
        chord = ta + (tb - ta) * (u - ua) / (ub - ua)
        assert np.max(np.abs(t - chord)) > 0.1


def test_missing_proton_gives_empty_row():
    mask = _ball_mask((20, 20, 6), 5.0)
    geo = _geo(shape=(20, 20, 6), mask=mask)
    h = _one_proton(0.0, t=9.0, v=0.0)
    st, ok, _ = O.prepare(geo, h)
    assert not ok[0]
    rp, j, ln, _ = O.rows(geo, h)
    assert rp.tolist() == [0, 0] and j.size == 0


# --------------------------------------------------------------------------
# DROP (Sec. IV-B)
# --------------------------------------------------------------------------

def _random_system(m=60, n=40, nnz_row=6, seed=0):
    rng = np.random.default_rng(seed)
    rows, cols, vals = [], [], []
    for i in range(m):
        js = rng.choice(n, size=nnz_row, replace=False)
        rows += [i] * nnz_row
        cols += js.tolist()
        vals += rng.uniform(0.1, 1.7, nnz_row).tolist()
    A = sp.csr_matrix((vals, (rows, cols)), shape=(m, n))
    xs = rng.uniform(0.3, 1.6, n)
    return A, xs


def test_drop_block_one_is_kaczmarz():
    A, xs = _random_system()
    b = A @ xs
    x0 = np.ones(A.shape[1])
    got = O.drop(A, b, iters=3, lam=0.7, block=1, x0=x0)
    x = x0.copy()
    Ad = A.toarray()
    for _ in range(3):
        for i in range(A.shape[0]):
            a = Ad[i]
            x = x + 0.7 * (b[i] - a @ x) / (a @ a) * a
    assert np.allclose(got, x, rtol=0, atol=1e-12)


def test_drop_single_block_is_simultaneous_sart_form():
    A, xs = _random_system(seed=1)
    rng = np.random.default_rng(1)
    b = A @ xs + rng.normal(0, 0.01, A.shape[0])
    x0 = np.full(A.shape[1], 0.9)
    got = O.drop(A, b, iters=1, lam=1.3, block=A.shape[0], x0=x0)
    W = 1.0 / np.asarray(A.multiply(A).sum(axis=1)).ravel()
    s = np.asarray((A != 0).sum(axis=0)).ravel()
    upd = A.T @ (W * (b - A @ x0))
    want = x0 + 1.3 * np.where(s > 0, upd / np.maximum(s, 1), 0.0)
    assert np.allclose(got, want, rtol=0, atol=1e-12)


def test_drop_blocks_run_in_order_and_each_block_is_fejer_monotone():
    A, xs = _random_system(m=90, n=50, nnz_row=8, seed=2)
    b = A @ xs
    x = np.ones(A.shape[1])
    B = 16
    whole = O.drop(A, b, iters=1, lam=1.8, block=B, x0=x)
    for t0 in range(0, A.shape[0], B):
        Ab = A[t0:t0 + B]
        xn = O.drop(Ab, b[t0:t0 + B], iters=1, lam=1.8, block=B, x0=x)
        s = np.asarray((Ab != 0).sum(axis=0)).ravel().astype(float)
        # error in the norm weighted by s_j (the inverse of DROP's diagonal) never grows
        e0 = np.sum(s * (x - xs) ** 2)
        e1 = np.sum(s * (xn - xs) ** 2)
        assert e1 <= e0 * (1 + 1e-12)
        assert np.array_equal(xn[s == 0], x[s == 0])
        x = xn
    assert np.allclose(x, whole, rtol=0, atol=1e-12)


def test_drop_consistent_data_fixed_point_and_convergence():
    A, xs = _random_system(m=200, n=40, nnz_row=7, seed=3)
    b = A @ xs
    assert np.allclose(O.drop(A, b, 2, 1.0, 32, xs), xs, atol=1e-12)
    x = np.ones(A.shape[1])
    errs = []
    for _ in range(8):
        x = O.drop(A, b, 1, 1.0, 1, x)
        errs.append(np.linalg.norm(x - xs))
    assert all(e1 <= e0 + 1e-12 for e0, e1 in zip(errs, errs[1:]))
    assert errs[-1] < 0.2 * np.linalg.norm(np.ones(A.shape[1]) - xs)


def _proton_system(n=4000):
    """Rows of synthetic protons through the tiny phantom, and its RSP."""
    cfg = synth.scaled(synth.CONFIGS["tiny"], n)
    rsp, hull = synth.phantom(cfg)
    hist = synth.to_numpy(synth.histories(cfg, "cpu", rsp=rsp))
    geo = O.Geometry(cfg.shape, (cfg.voxel,) * 3, cfg.origin, mask=hull.numpy())
    rowptr, j, ln, _ = O.rows(geo, hist)
    return O.csr(rowptr, j, ln, geo.n_vox), rowptr, j, ln, rsp.numpy() * hull.numpy(), hull.numpy()


def test_proton_rows_adjoint_identity():
    # <A x, y> = <x, A^T y> for the oracle's forward and adjoint of proton rows,
    # and A^T y equals the row-by-row accumulation of y_i a_ij
    A, rowptr, j, ln, xt, hull = _proton_system(2000)
    rng = np.random.default_rng(7)
    x = rng.uniform(0.2, 1.5, A.shape[1])
    y = rng.normal(size=A.shape[0])
    ax, aty = O.forward(A, x), O.adjoint(A, y)
    assert abs(ax @ y - x @ aty) <= 1e-12 * np.abs(ax) @ np.abs(y)
    acc = np.zeros(A.shape[1])
    for i in range(A.shape[0]):
        for e in range(rowptr[i], rowptr[i + 1]):
            acc[j[e]] += y[i] * ln[e]
    assert np.allclose(aty, acc, rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("lam,block", [(1.0, 4000), (0.5, 400), (1.0, 100), (0.5, 1)])
def test_drop_residual_falls_monotonically_on_noise_free_proton_data(lam, block):
    # b = A x_true from the oracle's own rows: every DROP iteration lowers ||A x - b||
    A, _, _, _, xt, hull = _proton_system()
    b = A @ xt
    x = hull.astype(np.float64)
    res = [np.linalg.norm(A @ x - b)]
    for _ in range(6):
        x = O.drop(A, b, 1, lam, block, x)
        res.append(np.linalg.norm(A @ x - b))
    assert all(r1 < r0 for r0, r1 in zip(res, res[1:])), res
    assert res[-1] < 0.5 * res[0]


def test_drop_skips_empty_rows_and_untouched_voxels():
    A = sp.csr_matrix(np.array([[0.0, 0.0, 0.0], [1.0, 0.0, 0.5]]))
    x = O.drop(A, np.array([5.0, 2.0]), 1, 1.0, 2, np.array([1.0, 1.0, 1.0]))
    r = (2.0 - 1.5) / 1.25
    assert np.allclose(x, [1.0 + r * 1.0, 1.0, 1.0 + r * 0.5])


# --------------------------------------------------------------------------
# Total variation
# --------------------------------------------------------------------------

def test_tv_gradient_matches_central_differences():
    rng = np.random.default_rng(5)
    shape = (5, 4, 3)
    x = rng.normal(size=60)
    v, g = O.tv(x, shape, eps=1e-3)
    h = 1e-6
    fd = np.array([(O.tv(x + h * e, shape, 1e-3)[0] - O.tv(x - h * e, shape, 1e-3)[0]) / (2 * h)
                   for e in np.eye(60)])
    assert np.allclose(g, fd, atol=1e-6)


def test_tv_closed_forms():
    shape = (6, 5, 4)
    assert np.isclose(O.tv(np.full(120, 2.5), shape, eps=1e-6)[0], 120 * 1e-6)
    step = np.zeros((4, 5, 6))
    step[:, :, 3:] = 1.0
    v, _ = O.tv(step.reshape(-1), shape, eps=1e-9)
    assert abs(v - 4 * 5 * 1.0) < 1e-6


def test_csr_leaves_path_order_rows_untouched():
    # building A must not reorder the caller's path-order rows
    rowptr = np.array([0, 3], dtype=np.int64)
    j = np.array([5, 1, 3], dtype=np.int32)
    ln = np.array([0.5, 0.25, 0.75])
    A = O.csr(rowptr, j, ln, 8)
    assert j.tolist() == [5, 1, 3] and ln.tolist() == [0.5, 0.25, 0.75]
    assert A.indices.tolist() == [1, 3, 5] and A.data.tolist() == [0.25, 0.75, 0.5]


def test_walk_consecutive_segments_share_their_vertex():
    # samples every 0.8 mm along x on a 1.6 mm grid put every other vertex on a
    # face (up to rounding); the walk must still move monotonically in x
    geo = _geo(shape=(40, 4, 4), voxel=(1.6, 1.25, 0.8), origin=(-33.0, -2.5, -1.6))
    xs = -26.6 + 0.8 * np.arange(67)
    pts = np.stack([xs, np.full_like(xs, 0.3), np.full_like(xs, 0.1)], axis=1)
    j, ln, _ = O.walk(geo, pts)
    ix = j % 40
    assert np.all(np.diff(ix) == 1), ix
    assert np.all(ln[1:-1] > 1.5)


def test_hull_entry_conditioning_of_the_crossed_face():
    # a line nearly parallel to the z faces entering the hull through one of
    # them: conditioning |D| / |D_z| (how far a position error moves the
    # crossing along the line); through an x face head on: about 1
    shape = (20, 20, 10)
    geo_z = _geo(shape=shape, origin=(-10.0, -10.0, -5.0),
                 mask=(np.arange(10)[:, None, None] >= 5).repeat(20, 1).repeat(20, 2).astype(np.uint8))
    D = np.array([1.0, 0.0, 0.02])
    hit, s, m, c = O.hull_entry(geo_z, [-9.9, 0.1, -0.15], D, 30.0, with_cond=True)
    assert hit and abs(s - 7.5) < 1e-12
    assert abs(c - np.linalg.norm(D) / 0.02) < 1e-9
    geo_x = _geo(shape=shape, origin=(-10.0, -10.0, -5.0),
                 mask=(np.arange(20)[None, None, :] >= 12).repeat(10, 0).repeat(20, 1).astype(np.uint8))
    hit, s, m, c = O.hull_entry(geo_x, [-9.9, 0.1, 0.15], D, 30.0, with_cond=True)
    assert hit and abs(s - 11.9) < 1e-12 and abs(c - np.linalg.norm(D)) < 1e-12
    # a line that starts inside its first hull voxel crosses no face: 1
    hit, s, m, c = O.hull_entry(geo_x, [2.5, 0.1, 0.15], D, 30.0, with_cond=True)
    assert hit and s == 0.0 and c == 1.0
