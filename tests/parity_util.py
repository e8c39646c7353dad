"""Shared helpers of the GPU parity tests: seeded scans, oracle results, comparisons."""
from __future__ import annotations

import functools

import numpy as np
import torch

import oracle as O
import synth
from oracle.compare import (CHORD_TOL_MM, MLP_TOL_MM, NEAR_FACE_MM, POS_ERR_MM, Exclusion,  # noqa: F401
                            chord_tol, near_face, solve_parity)


@functools.lru_cache(maxsize=8)
def scan(name: str, n: int | None = None):
    """(cfg, rsp, hull, host histories float32) of a workload, n protons (cached)."""
    cfg = synth.CONFIGS[name]
    if n is not None and n != cfg.n_protons:
        cfg = synth.scaled(cfg, n)
    rsp, hull = synth.phantom(cfg)
    hist = synth.to_numpy(synth.histories(cfg, "cpu", rsp=rsp))
    return cfg, rsp.numpy(), hull.numpy(), hist


def geometry(cfg, hull, **kw):
    return O.Geometry(cfg.shape, (cfg.voxel,) * 3, cfg.origin, mask=hull, **kw)


@functools.lru_cache(maxsize=8)
def oracle_rows(name: str, n: int | None = None):
    cfg, rsp, hull, hist = scan(name, n)
    geo = geometry(cfg, hull)
    rowptr, j, ln, margin, cond = O.rows(geo, hist, with_cond=True)
    A = O.csr(rowptr, j, ln, geo.n_vox)
    return geo, rowptr, j, ln, margin, A, cond


def context(cfg, hull, hist, device=0):
    import paper_1802_01070_b300 as pct
    ctx = pct.Context(cfg.shape, cfg.voxel, cfg.origin, hull=hull, device=device)
    dev = torch.device("cuda", device)
    ctx.load_histories({k: torch.from_numpy(np.ascontiguousarray(v)).to(dev) for k, v in hist.items()})
    return ctx


def compare_rows(gidx, glen, gnnz, rowptr, j, ln, margin, cond=None, dL=None,
                 chord_tol=CHORD_TOL_MM):
    """Compare GPU rows with the oracle's.  Returns (n_rows, n_excused, worst chord diff, bad).

    Voxel index sequences must be identical; a row may differ only when the
    oracle reports a crossing within NEAR_FACE_MM of a voxel face (margin).
    Chords of matching rows agree within chord_tol plus POS_ERR_MM times the
    row's crossing conditioning (a crossing nearly parallel to its face moves
    along the path by the sideways error over the sine of the angle).  An
    excused row's total chord length agrees up to its hull-depth difference dL.
    """
    n = gnnz.shape[0]
    excused = 0
    worst = 0.0
    bad = []
    for i in range(n):
        a, b = rowptr[i], rowptr[i + 1]
        oj, ol = j[a:b], ln[a:b]
        k = int(gnnz[i])
        gj, gl = gidx[i, :k], glen[i, :k]
        tol = chord_tol + (POS_ERR_MM * cond[i] if cond is not None else 0.0)
        if k == oj.size and np.array_equal(gj, oj):
            d = float(np.max(np.abs(gl - ol))) if k else 0.0
            worst = max(worst, d)
            if d > tol:
                bad.append((i, "chord", d))
            continue
        if near_face(margin[i], cond[i] if cond is not None else 0.0):
            excused += 1
            if dL is not None:
                dtot = abs(float(gl.sum()) - float(ol.sum()))
                if dtot > tol + dL[i]:
                    bad.append((i, "excused-row length", dtot))
            continue
        bad.append((i, "sequence", float(margin[i])))
    return n, excused, worst, bad


def gpu_exclusion(ctx, rowptr, j, ln, margin, cond, block, first=0, count=None, chunk=8192, x=None, b=None):
    """The voxels the comparison rule of ``oracle.compare`` leaves out, for the
    protons [first, first + count) loaded in ``ctx`` against the oracle's CSR
    rows of the same protons (rowptr indexed from ``first``), DROP blocks of
    ``block`` rows counted from ``first``.  For a single block step from the
    iterate ``x`` with measurements ``b`` (of those protons) the residual part
    of the rule applies too."""
    n = ctx.n - first if count is None else count
    ex = Exclusion(ctx.n_vox, block, x=x, b=b)
    for a in range(0, n, chunk):
        k = min(n, a + chunk) - a
        _, _, nnz = ctx.rows(first + a, k, max_nnz=0)
        W = max(int(nnz.max().item()), 1)
        gidx, glen, gnnz = ctx.rows(first + a, k, max_nnz=W)
        e0, e1 = int(rowptr[a]), int(rowptr[a + k])
        ex.add(a, gidx.cpu().numpy(), glen.cpu().numpy(), gnnz.cpu().numpy(),
               rowptr[a:a + k + 1] - rowptr[a], j[e0:e1], ln[e0:e1], margin[a:a + k], cond[a:a + k])
    return ex.finish()
