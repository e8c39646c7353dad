"""Pins of the FBP oracle (oracle/fbp.py) against things other than itself.

CPU only.  The ramp filter's response to a sinusoid (it must multiply a
frequency f by |f|), the reconstruction of a uniform disk from its analytic
projections, where an impulse in one sinogram bin lands when back-projected,
the per-bin means against a Python loop, and a disk reconstructed end to end
from straight synthetic protons.
"""
import math

import numpy as np
import pytest

from oracle import fbp as F


@pytest.mark.parametrize("tau,f", [(1.0, 0.05), (1.0, 0.2), (1.0, 0.45), (0.5, 0.3), (0.5, 0.9)])
def test_ramp_filter_multiplies_a_sinusoid_by_its_frequency(tau, f):
    # Kak-Slaney kernel: its DTFT is |f| for |f| <= 1 / (2 tau), f in cycles/mm
    n = 4001
    m = np.arange(n) - n // 2
    for phase in (0.0, 0.7):
        p = np.cos(2 * math.pi * f * m * tau + phase)
        q = F.ramp_filter(p[None, :], tau)[0]
        c = slice(n // 2 - 20, n // 2 + 21)
        assert np.allclose(q[c], f * p[c], atol=2e-3 * f + 1e-4 / tau)
    # a constant row has no interior response
    q = F.ramp_filter(np.ones((1, n)), tau)[0]
    assert abs(q[n // 2]) < 1e-3 / tau


def _disk_sino(p, R, rho, cx, cy):
    t = p.t_min + (np.arange(p.n_t) + 0.5) * p.dt
    sino = np.zeros((p.n_angle, p.n_v, p.n_t))
    for a in range(p.n_angle):
        phi = a * p.angle_step
        tc = -cx * math.sin(phi) + cy * math.cos(phi)
        d = t - tc
        sino[a, :, :] = np.where(np.abs(d) < R, 2 * rho * np.sqrt(np.maximum(R * R - d * d, 0)), 0.0)
    return sino


def test_uniform_disk_from_analytic_projections():
    p = F.FbpParams(n_angle=180, angle_step=2 * math.pi / 180, n_t=200, t_min=-80.0, dt=0.8,
                    n_v=1, v_min=-2.0, dv=4.0)
    R, rho, cx, cy = 30.0, 1.3, 5.0, -3.0
    q = F.ramp_filter(_disk_sino(p, R, rho, cx, cy), p.dt)
    shape, vox, org = (100, 100, 1), (1.0, 1.0, 1.0), (-50.0, -50.0, -0.5)
    img = F.backproject(q, p, shape, vox, org).reshape(100, 100)
    xc = org[0] + np.arange(100) + 0.5
    X, Y = np.meshgrid(xc, xc)
    r = np.hypot(X - cx, Y - cy)
    inside, outside = r < 0.8 * R, (r > 1.3 * R) & (r < 45)
    assert abs(img[inside].mean() - rho) < 0.002 * rho
    assert np.max(np.abs(img[inside] - rho)) < 0.01 * rho
    # outside: no offset, only the streaks of a finite number of views
    assert abs(img[outside].mean()) < 0.002 * rho
    assert np.abs(img[outside]).mean() < 0.03 * rho


def test_impulse_back_projects_to_a_strip_at_its_offset():
    # one non-zero bin (angle a0, bin k0) back-projects onto the voxels whose
    # centres lie within one bin of the line t = t_k0 at that angle, with the
    # linear-interpolation weight, pi / n_angle at the centre line
    n_angle = 8
    p = F.FbpParams(n_angle=n_angle, angle_step=2 * math.pi / n_angle, n_t=20, t_min=-10.0, dt=1.0,
                    n_v=1, v_min=-1.0, dv=2.0)
    shape, vox, org = (20, 20, 1), (1.0, 1.0, 1.0), (-10.0, -10.0, -0.5)
    xc = org[0] + np.arange(20) + 0.5
    X, Y = np.meshgrid(xc, xc)              # rows y, columns x
    for a0, k0 in ((0, 13), (2, 6), (4, 13)):
        q = np.zeros((n_angle, 1, p.n_t))
        q[a0, 0, k0] = 1.0
        img = F.backproject(q, p, shape, vox, org).reshape(20, 20)
        tk = p.t_min + (k0 + 0.5) * p.dt
        phi = a0 * p.angle_step
        t = -X * math.sin(phi) + Y * math.cos(phi)
        want = (math.pi / n_angle) * np.maximum(1.0 - np.abs(t - tk) / p.dt, 0.0)
        assert np.allclose(img, want, atol=1e-12)
        if a0 == 0:                          # phi = 0: t = y, a row of voxels
            assert np.allclose(img[np.abs(Y - tk) < 1e-9], math.pi / n_angle)
        if a0 == 2:                          # phi = pi/2: t = -x, a column
            assert np.allclose(img[np.abs(-X - tk) < 1e-9], math.pi / n_angle)


def _proton(phi, t_in, t_out, z_in, z_out, wepl, U=100.0):
    c, s = math.cos(phi), math.sin(phi)
    return {"in_x": -U * c - t_in * s, "in_y": -U * s + t_in * c, "in_z": z_in,
            "out_x": U * c - t_out * s, "out_y": U * s + t_out * c, "out_z": z_out,
            "theta_in": 0.0, "theta_out": 0.0, "psi_in": 0.0, "psi_out": 0.0, "phi": phi, "wepl": wepl}


def test_sinogram_means_match_a_per_bin_loop():
    rng = np.random.default_rng(3)
    p = F.FbpParams(n_angle=6, angle_step=2 * math.pi / 6, n_t=10, t_min=-10.0, dt=2.0, n_v=3,
                    v_min=-3.0, dv=2.0)
    prot = [_proton(int(rng.integers(0, 6)) * p.angle_step, rng.uniform(-12, 12), rng.uniform(-12, 12),
                    rng.uniform(-4, 4), rng.uniform(-4, 4), rng.uniform(10, 200)) for _ in range(3000)]
    h = {k: np.array([q[k] for q in prot], dtype=np.float32) for k in prot[0]}
    cnt, mean = F.sinogram(h, p)
    acc = {}
    # per-bin loop from the float32 histories
    phi = h["phi"].astype(np.float64)
    for i in range(len(prot)):
        c, s = math.cos(phi[i]), math.sin(phi[i])
        u0 = float(h["in_x"][i]) * c + float(h["in_y"][i]) * s
        t0 = -float(h["in_x"][i]) * s + float(h["in_y"][i]) * c
        u1 = float(h["out_x"][i]) * c + float(h["out_y"][i]) * s
        t1 = -float(h["out_x"][i]) * s + float(h["out_y"][i]) * c
        w = -u0 / (u1 - u0)
        t = t0 + w * (t1 - t0)
        v = float(h["in_z"][i]) + w * (float(h["out_z"][i]) - float(h["in_z"][i]))
        a = int(math.floor(phi[i] / p.angle_step + 0.5)) % p.n_angle
        kt = math.floor((t - p.t_min) / p.dt)
        kv = math.floor((v - p.v_min) / p.dv)
        if 0 <= kt < p.n_t and 0 <= kv < p.n_v:
            acc.setdefault((a, kv, kt), []).append(float(h["wepl"][i]))
    want = np.zeros_like(mean)
    wcnt = np.zeros_like(cnt)
    for (a, kv, kt), ws in acc.items():
        want[a, kv, kt] = sum(ws) / len(ws)
        wcnt[a, kv, kt] = len(ws)
    assert np.array_equal(cnt, wcnt)
    assert np.allclose(mean, want, rtol=1e-13, atol=0)


def test_disk_from_straight_protons_end_to_end():
    # protons that travel straight (no scattering) through a water disk of
    # radius 25 mm: WEPL = the chord length; the FBP image is ~1 inside
    rng = np.random.default_rng(8)
    n_angle, R = 90, 25.0
    p = F.FbpParams(n_angle=n_angle, angle_step=2 * math.pi / n_angle, n_t=80, t_min=-40.0, dt=1.0,
                    n_v=1, v_min=-5.0, dv=10.0)
    prot = []
    for i in range(90 * 2000):
        a = i % n_angle
        t = rng.uniform(-40, 40)
        z = rng.uniform(-4, 4)
        w = 2 * math.sqrt(R * R - t * t) if abs(t) < R else 0.0
        prot.append(_proton(a * p.angle_step, t, t, z, z, w))
    h = {k: np.array([q[k] for q in prot], dtype=np.float32) for k in prot[0]}
    shape, vox, org = (60, 60, 1), (1.0, 1.0, 1.0), (-30.0, -30.0, -0.5)
    img = F.fbp(h, p, shape, vox, org).reshape(60, 60)
    xc = org[0] + np.arange(60) + 0.5
    X, Y = np.meshgrid(xc, xc)
    r = np.hypot(X, Y)
    assert abs(img[r < 20].mean() - 1.0) < 0.002
    assert np.max(np.abs(img[r < 20] - 1.0)) < 0.03
    assert np.abs(img[r > 28]).mean() < 0.03
