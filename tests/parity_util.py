"""Shared helpers of the GPU parity tests: seeded scans, oracle results, comparisons."""
from __future__ import annotations

import functools

import numpy as np
import torch

import oracle as O
import synth

NEAR_FACE_MM = 1e-4     # crossings this close to a voxel face may legitimately differ (FP32 vs FP64)
MLP_TOL_MM = 1e-3       # MLP point tolerance
CHORD_TOL_MM = 2e-3     # chord tolerance (difference of two MLP-derived crossings)
POS_ERR_MM = 1e-5       # sideways position error of the FP32 path (MLP points agree to ~6e-6 mm)


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
        if margin[i] < NEAR_FACE_MM:
            excused += 1
            if dL is not None:
                dtot = abs(float(gl.sum()) - float(ol.sum()))
                if dtot > tol + dL[i]:
                    bad.append((i, "excused-row length", dtot))
            continue
        bad.append((i, "sequence", float(margin[i])))
    return n, excused, worst, bad


def structure_diff_voxels(gidx, gnnz, rowptr_o, j_o, block, n_vox):
    """Voxels whose DROP count s_j differs between the GPU rows and the oracle's
    rows in at least one block.

    s_j counts the rows of a block with a_ij > 0, so a grazing chord that one
    side resolves and the other does not (a near-face case) changes s_j by one.
    gidx/gnnz: GPU rows (visits in path order; the GPU counts each visit, so a
    near-face return to a voxel counts twice there); rowptr_o/j_o: oracle rows
    in path order (counted once per row and voxel).
    """
    m = gnnz.shape[0]
    blk_rows = np.arange(m) // block
    k = np.minimum(gnnz, gidx.shape[1])
    g_rows = np.repeat(np.arange(m), k)
    g_j = np.concatenate([gidx[i, :k[i]] for i in range(m)]) if m else np.zeros(0, np.int64)
    o_rows = np.repeat(np.arange(m), np.diff(rowptr_o))
    # one count per (row, voxel) on the oracle side, as DROP defines s_j
    ok = np.unique(o_rows.astype(np.int64) * n_vox + j_o)
    o_rows_u, o_j_u = ok // n_vox, ok % n_vox
    nb = int(blk_rows[-1]) + 1 if m else 0
    co = np.bincount(blk_rows[o_rows_u] * n_vox + o_j_u, minlength=nb * n_vox)
    # the GPU scatter counts every visit
    cg = np.bincount(blk_rows[g_rows] * n_vox + g_j.astype(np.int64), minlength=nb * n_vox)
    diff = (co != cg).reshape(nb, n_vox).any(axis=0) if nb else np.zeros(n_vox, bool)
    return diff


def solve_parity(xg, xo, hull, diff_vox):
    """(max rel err on hull voxels with identical row structure, count of other
    hull voxels, max rel err over all hull voxels, fraction within 1e-3)."""
    hm = hull.astype(bool)
    rel = np.abs(xg - xo) / np.maximum(np.abs(xo), 1e-30)
    clean = hm & ~diff_vox
    return (float(rel[clean].max()) if clean.any() else 0.0, int((hm & diff_vox).sum()),
            float(rel[hm].max()), float((rel[hm] <= 1e-3).mean()))


def chord_diff_voxels(gidx, glen, gnnz, rowptr_o, j_o, ln_o, n_vox, tol=CHORD_TOL_MM):
    """Voxels crossed by a row whose GPU and oracle chords differ by more than
    tol (a grazing crossing resolved differently in FP32 and FP64), or by a
    row whose voxel sequence differs."""
    m = gnnz.shape[0]
    out = np.zeros(n_vox, bool)
    for i in range(m):
        a, b = rowptr_o[i], rowptr_o[i + 1]
        k = int(gnnz[i])
        gj, gl = gidx[i, :k], glen[i, :k]
        oj, ol = j_o[a:b], ln_o[a:b]
        if k == oj.size and np.array_equal(gj, oj):
            bad = np.abs(gl - ol) > tol
            out[oj[bad]] = True
        else:
            # sequences differ (near-face row): flag voxels whose chord sum differs
            vox = np.union1d(gj, oj)
            sg = np.zeros(vox.size)
            so = np.zeros(vox.size)
            np.add.at(sg, np.searchsorted(vox, gj), gl)
            np.add.at(so, np.searchsorted(vox, oj), ol)
            out[vox[np.abs(sg - so) > tol]] = True
    return out
