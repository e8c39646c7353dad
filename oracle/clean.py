"""FP64 oracle of the data-cleaning step -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU legs of ``bench.py``
use this module; the product library never imports it and it imports nothing
from the product library.

What it computes.  The paper reduces its scans before the solve by "data
cleaning techniques (e.g. identifying and removing statistical outliers)"
(Sec. IV-A: 116 million histories become 21 million, 261 million become 78
million) and gives no further detail.  The reading taken here, the usual one
for proton-CT list-mode data:

* Every proton falls into one bin of (gantry angle, t, v): the angle bin is the
  nearest multiple of ``angle_step`` (modulo ``n_angle``), t and v are the
  lateral and vertical positions where the straight chord between the entry
  and exit tracker points crosses depth u = 0 of the beam frame of its gantry
  angle (t = (t_in + t_out) / 2, v = (z_in + z_out) / 2 when the trackers sit
  at -U and +U), binned from ``t_min`` / ``v_min`` in steps ``dt`` / ``dv``.
  Protons outside the ``n_t`` x ``n_v`` bins are removed.
* In each bin, three quantities are tested: the WEPL, the change of the t-u
  plane angle theta_out - theta_in and the change of the v-u plane angle
  psi_out - psi_in.  For each, the bin's mean mu and population standard
  deviation sigma (sum of squared deviations over the bin count, two passes).
* A proton is kept when all three satisfy |q - mu| <= k_sigma * sigma.

Everything is FP64 from the float32 histories.  Library primitives (numpy
bincount for the per-bin sums) are steps of the definition; there is no
reordering beyond that.

Parity status: pinned by tests/test_oracle_clean.py (a pure-Python per-bin
loop on small scans, closed-form bins, and the removal of planted outliers).
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np


@dataclass(frozen=True)
class CleanParams:
    n_angle: int        # angle bins over a full turn
    angle_step: float   # rad, width of an angle bin
    n_t: int
    t_min: float        # mm, lower edge of t bin 0
    dt: float           # mm
    n_v: int
    v_min: float        # mm
    dv: float           # mm
    k_sigma: float = 3.0


def bin_coordinates(hist):
    """(angle coordinate phi / step, t, v) per proton in FP64: the chord's
    lateral and vertical position at depth u = 0."""
    x0 = np.asarray(hist["in_x"], np.float64)
    y0 = np.asarray(hist["in_y"], np.float64)
    z0 = np.asarray(hist["in_z"], np.float64)
    x1 = np.asarray(hist["out_x"], np.float64)
    y1 = np.asarray(hist["out_y"], np.float64)
    z1 = np.asarray(hist["out_z"], np.float64)
    phi = np.asarray(hist["phi"], np.float64)
    c, s = np.cos(phi), np.sin(phi)
    u0, t0 = x0 * c + y0 * s, -x0 * s + y0 * c
    u1, t1 = x1 * c + y1 * s, -x1 * s + y1 * c
    # chord parameter of depth u = 0 (u0 < 0 < u1 for a proton crossing the
    # rotation axis plane); at u0 = -u1 this is the midpoint
    w = -u0 / (u1 - u0)
    t = t0 + w * (t1 - t0)
    v = z0 + w * (z1 - z0)
    return phi, t, v


def bin_index(hist, p: CleanParams):
    """Bin of every proton (int64, -1 when outside the t or v bins)."""
    phi, t, v = bin_coordinates(hist)
    a = np.floor(phi / p.angle_step + 0.5).astype(np.int64) % p.n_angle
    kt = np.floor((t - p.t_min) / p.dt)
    kv = np.floor((v - p.v_min) / p.dv)
    ok = (kt >= 0) & (kt < p.n_t) & (kv >= 0) & (kv < p.n_v)
    kt = np.where(ok, kt, 0).astype(np.int64)
    kv = np.where(ok, kv, 0).astype(np.int64)
    b = (a * p.n_v + kv) * p.n_t + kt
    return np.where(ok, b, -1)


def quantities(hist):
    """(WEPL, theta_out - theta_in, psi_out - psi_in) in FP64, shape (3, n)."""
    w = np.asarray(hist["wepl"], np.float64)
    dth = np.asarray(hist["theta_out"], np.float64) - np.asarray(hist["theta_in"], np.float64)
    dps = np.asarray(hist["psi_out"], np.float64) - np.asarray(hist["psi_in"], np.float64)
    return np.stack([w, dth, dps])


def bin_stats(hist, p: CleanParams):
    """(bin per proton, count per bin, mean (3, nbins), sigma (3, nbins))."""
    b = bin_index(hist, p)
    nb = p.n_angle * p.n_v * p.n_t
    q = quantities(hist)
    inb = b >= 0
    cnt = np.bincount(b[inb], minlength=nb).astype(np.float64)
    safe = np.maximum(cnt, 1.0)
    mean = np.stack([np.bincount(b[inb], weights=q[k][inb], minlength=nb) / safe for k in range(3)])
    dev2 = np.stack([np.bincount(b[inb], weights=(q[k][inb] - mean[k][b[inb]]) ** 2, minlength=nb)
                     for k in range(3)])
    sigma = np.sqrt(dev2 / safe)
    return b, cnt, mean, sigma


def clean(hist, p: CleanParams):
    """Keep mask (bool, n) and the per-proton relative margin to the nearest cut.

    ``margin`` is min over the three quantities of (k sigma - |q - mu|) /
    max(k sigma, |q - mu|): in [-1, 1], negative for a removed proton, 0 where
    both are 0, +inf for protons outside the bins.  Parity tests excuse
    protons whose margin is within rounding of 0.
    """
    b, cnt, mean, sigma = bin_stats(hist, p)
    q = quantities(hist)
    inb = b >= 0
    bb = np.where(inb, b, 0)
    lim = p.k_sigma * sigma[:, bb]
    dev = np.abs(q - mean[:, bb])
    keep = inb & np.all(dev <= lim, axis=0)
    scale = np.maximum(lim, dev)
    rel = np.where(scale > 0, (lim - dev) / np.where(scale > 0, scale, 1.0), 0.0)
    margin = np.where(inb, np.min(rel, axis=0), np.inf)
    return keep, margin
