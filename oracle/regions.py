"""FP64 oracle of the image regions of the paper's Algorithm 1 -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU legs of ``bench.py``
use this module; the product library never imports it and it imports nothing
from the product library.

What it computes (arXiv:1802.01070, Sec. III, Algorithm 1):
1. setupImageRegions: the z slices are split into ``n_regions`` core ranges
   [r nz / R, (r+1) nz / R) (integer division), each extended by ``halo``
   slices on both sides, clamped to the volume.  (The paper's example: 20
   slices, two regions 0-12 and 7-19, i.e. halo 3, cores 0-9 and 10-19.)
2. identifyProtonsPassingRegions: a proton with a hull path belongs to a
   region when the slices of both its hull entry point and its hull exit
   point lie in the region's extended range ("the image region entered to
   and exited from"), so that its path lies in the region's slab; protons
   that fit no region are not used (the paper sizes the overlap "for a 96%
   coverage").  A point on the grid's lowest or highest face counts in the
   first or last slice.
3./4. allocateMemoryForProtonsPerGPU, iterativelySolvePerGPU: each region is
   solved by DROP on its own, from the initial iterate's slab, with its
   protons' rows restricted to the region's extended slices (the path data of
   a row outside the slab is not part of that region's system).
5. selectSlice: the final volume takes each region's core slices.

Rows are the oracle's (``oracle.rows`` on the full volume: the same MLP path as
the single-region solve); DROP is ``oracle.drop``.  Readings: membership needs
both end points in the region (the other reading, either end point, gives a
region rows cut off at its slab with the full WEPL as right-hand side; its
system is inconsistent, and with a thin overlap DROP diverges); a row keeps
only the voxels of its region's slab (a path that bends out of the slab
between its end points loses that part).

Parity status: pinned by tests/test_oracle_regions.py (one region is the plain
solve, regions covering the whole volume reproduce it, the paper's example
slices, membership from the MLP polyline's end points, restricted rows).
"""
from __future__ import annotations

import numpy as np

import oracle as O


def regions(nz: int, n_regions: int, halo: int):
    """[(lo, hi, elo, ehi)] per region: core and extended slice ranges."""
    out = []
    for r in range(n_regions):
        lo, hi = r * nz // n_regions, (r + 1) * nz // n_regions
        out.append((lo, hi, max(0, lo - halo), min(nz, hi + halo)))
    return out


def entry_exit_slices(geo: "O.Geometry", hist):
    """(valid, slice of the hull entry point, slice of the hull exit point)."""
    st, valid, _ = O.prepare(geo, hist)
    oz, dz, nz = geo.origin[2], geo.voxel[2], geo.shape[2]
    s_in = np.clip(np.floor((st[:, 4] - oz) / dz), 0, nz - 1).astype(np.int64)
    s_out = np.clip(np.floor((st[:, 8] - oz) / dz), 0, nz - 1).astype(np.int64)
    return valid, s_in, s_out


def members(valid, s_in, s_out, elo: int, ehi: int):
    return valid & (s_in >= elo) & (s_in < ehi) & (s_out >= elo) & (s_out < ehi)


def restrict_rows(rowptr, j, ln, sel, plane: int, elo: int, ehi: int):
    """CSR rows of the selected protons, keeping the entries in slices
    [elo, ehi) re-indexed to the slab (j - elo * plane)."""
    rows = np.flatnonzero(sel)
    starts, ends = rowptr[rows], rowptr[rows + 1]
    counts = ends - starts
    idx = np.repeat(starts - np.concatenate([[0], np.cumsum(counts)[:-1]]), counts) + np.arange(counts.sum())
    jj, ll = j[idx].astype(np.int64), ln[idx]
    owner = np.repeat(np.arange(rows.size), counts)
    keep = (jj >= elo * plane) & (jj < ehi * plane)
    rp = np.zeros(rows.size + 1, dtype=np.int64)
    np.add.at(rp, owner[keep] + 1, 1)
    np.cumsum(rp, out=rp)
    return rp, (jj[keep] - elo * plane).astype(np.int32), ll[keep]


def solve(geo: "O.Geometry", hist, n_regions: int, halo: int, iters: int, lam: float, block: int, x0,
          rows=None):
    """Algorithm 1: (x, protons per region).  ``rows`` = (rowptr, j, ln) of the
    full volume if already computed."""
    nx, ny, nz = geo.shape
    plane = nx * ny
    if rows is None:
        rowptr, j, ln, _ = O.rows(geo, hist)
    else:
        rowptr, j, ln = rows
    valid, s_in, s_out = entry_exit_slices(geo, hist)
    b = np.asarray(hist["wepl"], np.float64)
    x0 = np.asarray(x0, np.float64)
    x = x0.copy()
    counts = []
    for lo, hi, elo, ehi in regions(nz, n_regions, halo):
        sel = members(valid, s_in, s_out, elo, ehi)
        counts.append(int(sel.sum()))
        n_sub = (ehi - elo) * plane
        xr = x0[elo * plane:ehi * plane].copy()
        if sel.any():
            rp, jr, lr = restrict_rows(rowptr, j, ln, sel, plane, elo, ehi)
            A = O.csr(rp, jr, lr, n_sub)
            xr = O.drop(A, b[sel], iters, lam, block, xr)
        x[lo * plane:hi * plane] = xr[(lo - elo) * plane:(hi - elo) * plane]
    return x, counts
