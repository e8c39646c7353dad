"""FP64 oracle of the filtered back-projection (FBP) initial iterate -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU legs of ``bench.py``
use this module; the product library never imports it and it imports nothing
from the product library.

What it computes.  The paper starts its iterative solve from "the FBP image as
the initial iterate" (Sec. I) and gives no further detail.  The reading taken
here is the textbook parallel-beam FBP (Kak and Slaney, Principles of
Computerized Tomographic Imaging, ch. 3) applied slice by slice to binned
list-mode proton data:

1. Sinogram: every proton falls into a bin (angle a, v bin l, t bin k) as in
   the data-cleaning step -- a = nearest multiple of angle_step (mod n_angle);
   t, v = where the straight chord between its entry and exit tracker points
   crosses depth u = 0 of its beam frame, k = floor((t - t_min) / dt),
   l = floor((v - v_min) / dv).  p[a, l, k] = mean WEPL of the bin's protons,
   0 for an empty bin; protons outside the bins are not used.
2. Ramp filter along t (the band-limited spatial kernel of the reference
   above, spacing tau = dt): h[0] = 1 / (4 tau^2), h[n] = 0 for even n != 0,
   h[n] = -1 / (pi^2 n^2 tau^2) for odd n;  q[k] = tau sum_m p[m] h[k - m]
   over the row's n_t bins (zero beyond them).
3. Back-projection: voxel centre (x, y, z) takes the slice l of z, and
   x_fbp = (pi / n_angle) sum_a q_a(t_a), t_a = -x sin(phi_a) + y cos(phi_a),
   phi_a = a angle_step, q_a(t) linear between the bin centres t_min +
   (k + 1/2) dt and 0 beyond the first and last centres.  (A full turn sees
   every line twice: the integral over [0, pi) is half the sum over the turn.)
4. Initial iterate: the FBP value inside the hull, 0 outside.

FP64 throughout; numpy bincount (the per-bin sums) and vectorised loops are
steps of the definition.

Parity status: pinned by tests/test_oracle_fbp.py (the filter's response to a
sinusoid, the analytic reconstruction of a uniform disk, the back-projector as
the adjoint of an independently written forward sampler, a per-bin loop).
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

from oracle.clean import bin_coordinates


@dataclass(frozen=True)
class FbpParams:
    n_angle: int
    angle_step: float   # rad
    n_t: int
    t_min: float        # mm
    dt: float           # mm
    n_v: int
    v_min: float        # mm
    dv: float           # mm


def sinogram(hist, p: FbpParams):
    """(count, mean WEPL), both shaped (n_angle, n_v, n_t), FP64."""
    phi, t, v = bin_coordinates(hist)
    a = np.floor(phi / p.angle_step + 0.5).astype(np.int64) % p.n_angle
    kt = np.floor((t - p.t_min) / p.dt)
    kv = np.floor((v - p.v_min) / p.dv)
    ok = (kt >= 0) & (kt < p.n_t) & (kv >= 0) & (kv < p.n_v)
    b = (a[ok] * p.n_v + kv[ok].astype(np.int64)) * p.n_t + kt[ok].astype(np.int64)
    nb = p.n_angle * p.n_v * p.n_t
    cnt = np.bincount(b, minlength=nb).astype(np.float64)
    s = np.bincount(b, weights=np.asarray(hist["wepl"], np.float64)[ok], minlength=nb)
    mean = np.where(cnt > 0, s / np.maximum(cnt, 1.0), 0.0)
    shape = (p.n_angle, p.n_v, p.n_t)
    return cnt.reshape(shape), mean.reshape(shape)


def ramp_kernel(n_t: int, tau: float):
    """h[n] for n = -(n_t - 1) .. n_t - 1 (index n + n_t - 1)."""
    n = np.arange(-(n_t - 1), n_t, dtype=np.float64)
    h = np.zeros_like(n)
    h[n == 0] = 1.0 / (4.0 * tau * tau)
    odd = (np.abs(n) % 2) == 1
    h[odd] = -1.0 / (math.pi ** 2 * n[odd] ** 2 * tau * tau)
    return h


def ramp_filter(sino, dt: float):
    """q[..., k] = dt sum_m sino[..., m] h[k - m] along the last axis."""
    n_t = sino.shape[-1]
    h = ramp_kernel(n_t, dt)
    # the n_t x n_t Toeplitz matrix H[k, m] = h[k - m]
    k = np.arange(n_t)
    H = h[(k[:, None] - k[None, :]) + n_t - 1]
    return dt * np.einsum("...m,km->...k", sino, H)


def backproject(q, p: FbpParams, shape, voxel, origin, voxels=None):
    """FBP values at voxel centres (all voxels in j order, or the given linear
    indices ``voxels``)."""
    nx, ny, nz = shape
    if voxels is None:
        voxels = np.arange(nx * ny * nz, dtype=np.int64)
    voxels = np.asarray(voxels, dtype=np.int64)
    ix = voxels % nx
    iy = (voxels // nx) % ny
    iz = voxels // (nx * ny)
    x = origin[0] + (ix + 0.5) * voxel[0]
    y = origin[1] + (iy + 0.5) * voxel[1]
    z = origin[2] + (iz + 0.5) * voxel[2]
    l = np.floor((z - p.v_min) / p.dv)
    okz = (l >= 0) & (l < p.n_v)
    l = np.where(okz, l, 0).astype(np.int64)
    out = np.zeros(voxels.size)
    for a in range(p.n_angle):
        phi = a * p.angle_step
        t = -x * math.sin(phi) + y * math.cos(phi)
        f = (t - p.t_min) / p.dt - 0.5        # position in units of bins from the first centre
        k0 = np.floor(f)
        w = f - k0
        k0 = k0.astype(np.int64)
        row = q[a]                            # (n_v, n_t)
        v0 = np.where((k0 >= 0) & (k0 < p.n_t), row[l, np.clip(k0, 0, p.n_t - 1)], 0.0)
        v1 = np.where((k0 + 1 >= 0) & (k0 + 1 < p.n_t), row[l, np.clip(k0 + 1, 0, p.n_t - 1)], 0.0)
        out += (1.0 - w) * v0 + w * v1
    out *= math.pi / p.n_angle
    return np.where(okz, out, 0.0)


def fbp(hist, p: FbpParams, shape, voxel, origin, hull=None, voxels=None):
    """The FBP initial iterate: FBP inside the hull (all of it when hull is
    None), 0 outside; at all voxels or the given ones."""
    _, mean = sinogram(hist, p)
    q = ramp_filter(mean, p.dt)
    img = backproject(q, p, shape, voxel, origin, voxels)
    if hull is not None:
        hm = np.asarray(hull).reshape(-1).astype(bool)
        sel = hm if voxels is None else hm[np.asarray(voxels, dtype=np.int64)]
        img = np.where(sel, img, 0.0)
    return img
