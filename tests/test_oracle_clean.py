"""Pins of the data-cleaning oracle (oracle/clean.py) against things other than itself.

CPU only.  A pure-Python loop over bins on small scans, a bin whose mean and
standard deviation are known in closed form, the chord geometry of the bin
coordinates, the wrap of the angle bins, and the removal of planted outliers.
"""
import math

import numpy as np
import pytest

from oracle import clean as C


def _proton(phi, t_in, t_out, z_in, z_out, wepl, th=(0.0, 0.0), ps=(0.0, 0.0), U=100.0, u_in=None,
            u_out=None):
    c, s = math.cos(phi), math.sin(phi)
    ui = -U if u_in is None else u_in
    uo = U if u_out is None else u_out
    return {"in_x": ui * c - t_in * s, "in_y": ui * s + t_in * c, "in_z": z_in,
            "out_x": uo * c - t_out * s, "out_y": uo * s + t_out * c, "out_z": z_out,
            "theta_in": th[0], "theta_out": th[1], "psi_in": ps[0], "psi_out": ps[1],
            "phi": phi, "wepl": wepl}


def _stack(protons):
    return {k: np.array([p[k] for p in protons], dtype=np.float32) for k in protons[0]}


P1 = C.CleanParams(n_angle=4, angle_step=math.pi / 2, n_t=4, t_min=-20.0, dt=10.0, n_v=2,
                   v_min=-10.0, dv=10.0, k_sigma=3.0)


def test_bin_coordinates_are_the_chord_at_depth_zero():
    # symmetric trackers: the chord crosses u = 0 at the mean of the tracker positions
    h = _stack([_proton(0.7, 3.0, 7.0, -2.0, 4.0, 100.0)])
    phi, t, v = C.bin_coordinates(h)
    assert abs(t[0] - 5.0) < 1e-5 and abs(v[0] - 1.0) < 1e-5
    # asymmetric trackers (u_in = -50, u_out = 150): a quarter of the way
    h = _stack([_proton(2.1, 4.0, 8.0, 0.0, 8.0, 100.0, u_in=-50.0, u_out=150.0)])
    _, t, v = C.bin_coordinates(h)
    assert abs(t[0] - 5.0) < 1e-5 and abs(v[0] - 2.0) < 1e-5


def test_angle_bins_round_to_the_nearest_step_and_wrap():
    step = 2 * math.pi / 180
    phis = [0.0, 17 * step, 17.4 * step, 17.6 * step, 2 * math.pi - 0.2 * step, 179 * step]
    p = C.CleanParams(n_angle=180, angle_step=step, n_t=1, t_min=-1e3, dt=2e3, n_v=1, v_min=-1e3, dv=2e3)
    h = _stack([_proton(f, 0.0, 0.0, 0.0, 0.0, 1.0) for f in phis])
    assert C.bin_index(h, p).tolist() == [0, 17, 17, 18, 0, 179]


def test_closed_form_bin():
    # one bin, WEPL 10, 10, 10, 10, 20: mean 12, population sigma 4; theta
    # changes of -1, 1, -1, 1, 0 mrad (mean 0, sigma 0.8944 mrad), psi the same
    ang = (-1e-3, 1e-3, -1e-3, 1e-3, 0.0)
    h = _stack([_proton(0.0, 1.0, 1.0, 1.0, 1.0, w, th=(0.0, a), ps=(0.0, a))
                for w, a in zip((10, 10, 10, 10, 20), ang)])
    b, cnt, mean, sigma = C.bin_stats(h, P1)
    k = b[0]
    assert np.all(b == k) and cnt[k] == 5
    assert mean[0, k] == 12.0 and abs(sigma[0, k] - 4.0) < 1e-15
    sd_a = math.sqrt(4 * float(np.float32(1e-3)) ** 2 / 5)
    assert abs(sigma[1, k] - sd_a) < 1e-15 and abs(sigma[2, k] - sd_a) < 1e-15
    keep, margin = C.clean(h, P1)                 # 3 sigma = 12 mm, 2.68 mrad: all kept
    assert keep.all()
    # relative margins: proton 0's tightest cut is its angle, 1 - 1 mrad / 3 sd_a;
    # proton 4's is its WEPL, 8 mm inside 12 mm (its angle change is the mean)
    a1 = float(np.float32(1e-3))
    assert abs(margin[0] - (1.0 - a1 / (3 * sd_a))) < 1e-12
    assert abs(margin[4] - (12.0 - 8.0) / 12.0) < 1e-12
    keep, margin = C.clean(h, C.CleanParams(**{**P1.__dict__, "k_sigma": 1.5}))   # 6 mm: the 20 goes
    assert keep.tolist() == [True, True, True, True, False]
    assert abs(margin[4] - (6.0 - 8.0) / 8.0) < 1e-12


def test_out_of_range_protons_are_removed():
    h = _stack([_proton(0.0, 1.0, 1.0, 1.0, 1.0, 10.0), _proton(0.0, 30.0, 30.0, 1.0, 1.0, 10.0),
                _proton(0.0, 1.0, 1.0, -30.0, -30.0, 10.0)])
    assert C.bin_index(h, P1).tolist()[1:] == [-1, -1]
    keep, margin = C.clean(h, P1)
    assert keep.tolist() == [True, False, False] and np.isinf(margin[1:]).all()


def _brute(h, p):
    """Per-bin loop in plain Python floats (independent of numpy's bincount)."""
    n = len(h["wepl"])
    phi, t, v = C.bin_coordinates(h)
    bins = {}
    for i in range(n):
        a = int(math.floor(float(phi[i]) / p.angle_step + 0.5)) % p.n_angle
        kt = math.floor((float(t[i]) - p.t_min) / p.dt)
        kv = math.floor((float(v[i]) - p.v_min) / p.dv)
        if 0 <= kt < p.n_t and 0 <= kv < p.n_v:
            bins.setdefault((a, kv, kt), []).append(i)
    q = [[float(h["wepl"][i]), float(h["theta_out"][i]) - float(h["theta_in"][i]),
          float(h["psi_out"][i]) - float(h["psi_in"][i])] for i in range(n)]
    keep = [False] * n
    for members in bins.values():
        mu = [sum(q[i][c] for i in members) / len(members) for c in range(3)]
        sd = [math.sqrt(sum((q[i][c] - mu[c]) ** 2 for i in members) / len(members)) for c in range(3)]
        for i in members:
            keep[i] = all(abs(q[i][c] - mu[c]) <= p.k_sigma * sd[c] for c in range(3))
    return np.array(keep)


@pytest.mark.parametrize("seed", [0, 1])
def test_matches_a_per_bin_python_loop(seed):
    rng = np.random.default_rng(seed)
    n = 4000
    prot = []
    for _ in range(n):
        a = int(rng.integers(0, 4))
        prot.append(_proton(a * math.pi / 2 + rng.normal(0, 0.05), rng.uniform(-22, 22),
                            rng.uniform(-22, 22), rng.uniform(-11, 11), rng.uniform(-11, 11),
                            rng.normal(150, 3) if rng.random() > 0.02 else rng.uniform(0, 300),
                            th=(rng.normal(0, 0.005), rng.normal(0, 0.01)),
                            ps=(rng.normal(0, 0.005), rng.normal(0, 0.01))))
    h = _stack(prot)
    keep, margin = C.clean(h, P1)
    want = _brute(h, P1)
    near = np.abs(margin) < 1e-12
    assert np.array_equal(keep[~near], want[~near])
    assert 0.8 * n < keep.sum() < n


def test_planted_outliers_are_removed():
    # Gaussian bins with a few protons moved by 10 sigma in WEPL or in angle
    rng = np.random.default_rng(5)
    prot, planted = [], []
    for i in range(6000):
        bad = i % 97 == 0
        w = rng.normal(200, 2.0) + (25.0 if bad and i % 2 else 0.0)
        dth = rng.normal(0, 0.004) + (0.06 if bad and not i % 2 else 0.0)
        prot.append(_proton(0.0, rng.uniform(-20, 20), 0.0, 0.0, 0.0, w, th=(0.0, dth)))
        planted.append(bad)
    h = _stack(prot)
    p = C.CleanParams(n_angle=1, angle_step=2 * math.pi, n_t=2, t_min=-10.0, dt=10.0, n_v=1,
                      v_min=-5.0, dv=10.0)
    keep, _ = C.clean(h, p)
    planted = np.array(planted)
    assert not keep[planted].any()
    # a clean Gaussian loses ~0.27 % per quantity beyond 3 sigma
    assert keep[~planted].mean() > 0.985
