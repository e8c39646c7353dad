"""GPU rows and reconstructions against the FP64 oracle -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` use this module.  It holds no reconstruction arithmetic: it
compares rows and volumes that the GPU path and the oracle produced
independently, and states the one rule by which a voxel is left out of an RSP
comparison.

Why voxels are left out at all: the GPU path computes paths in FP32 (positions
good to ~1e-5 mm), the oracle in FP64.  Where a crossing lies within 1e-4 mm of
a voxel face (the oracle reports each row's smallest such distance, its
``margin``), the two may resolve the crossing into different voxels, and DROP's
count s_j of a block (rows with a_ij > 0, Sec. IV-B) or a chord then differs.
A voxel whose DROP inputs differ cannot be expected to match.

The rule (one rule, for every test and the benchmark) has two parts.

Row correctness.  cond is a row's crossing conditioning (path length per unit
of travel across a crossed face): the FP32 path's position error POS_ERR_MM
moves a crossing nearly parallel to its face by about POS_ERR_MM x cond, along
the path and along the face.  The oracle flags a row when a crossing lies
within NEAR_FACE_MM + POS_ERR_MM x cond of another face (near_face).  A row it
does not flag must have the oracle's voxel sequence and every chord within
chord_tol(cond) = CHORD_TOL_MM + POS_ERR_MM x cond; a row that fails is
counted as ``unexcused``: a real disagreement, which the tests assert away.

Voxel exclusion.  A hull voxel j is left out of an RSP comparison when its DROP
inputs differ between the two sides:
  (a) count: s_j differs between the GPU rows (every visit counts, as the GPU
      scatter does) and the oracle's rows (one count per row and voxel) in
      some DROP block;
  (b) chord: some row crosses j with chords that differ by more than
      CHORD_TOL_MM (for a row whose voxel sequence differs: the row's summed
      chord in j).  On a grazing crossing a chord can be correct by the row
      rule and still differ by more than CHORD_TOL_MM, which moves that
      voxel's update;
  (c) residual (for one block step from a known iterate x, with the rows'
      measurements b): voxel j's update takes lambda a_ij r_i / s_j from every
      row i through it, and r_i = (b_i - a_i.x) / ||a_i||^2 depends on the whole
      row.  A row that differs somewhere -- most of all one whose hull entry
      point moved along a grazing tracker line, which shifts the whole path --
      changes r_i on voxels where its chords agree.  Each side's r_i is
      evaluated in FP64 from its own row and the same x; voxel j of row i is
      left out when a_ij |r_i(GPU) - r_i(oracle)| > RESID_TOL |x_j| (a tenth
      of the relative RSP tolerance; lambda <= 1 <= s_j makes it a bound on
      the move).
      Across several blocks x itself differs and (c) does not apply: such
      runs are compared by statistics over all hull voxels.
"""
from __future__ import annotations

import numpy as np

NEAR_FACE_MM = 1e-4     # crossings this close to a voxel face may legitimately differ
MLP_TOL_MM = 1e-3       # MLP point tolerance
CHORD_TOL_MM = 2e-3     # chord tolerance (difference of two MLP-derived crossings)
POS_ERR_MM = 4e-5       # position error of the FP32 path: MLP points agree with the oracle's to
                        # 6.5e-6 mm on the small scans and 3.3e-5 mm on the full-size ones
RESID_TOL = 1e-4        # largest relative move a_ij |delta r_i| / |x_j| of a voxel by a row's residual


def chord_tol(cond):
    """Chord tolerance of a row: CHORD_TOL_MM plus POS_ERR_MM times the row's
    crossing conditioning (a crossing nearly parallel to its face moves along
    the path by the sideways error over the sine of the angle)."""
    return CHORD_TOL_MM + POS_ERR_MM * np.asarray(cond, dtype=np.float64)


def near_face(margin, cond):
    """Rows the oracle flags: a crossing within NEAR_FACE_MM of another voxel
    face, widened by the distance POS_ERR_MM x cond by which the FP32 path's
    position error can move a grazing crossing along the face."""
    return np.asarray(margin) < NEAR_FACE_MM + POS_ERR_MM * np.asarray(cond, dtype=np.float64)


def compare_row_chunk(gidx, glen, gnnz, rowptr, j, ln, margin, cond):
    """Compare padded GPU rows (m x W) with the oracle's CSR rows of the same protons.

    Returns a dict: ``chord_vox`` (voxels excluded by chord, part (b)),
    ``unexcused`` (indices of rows that fail the row rule without an oracle
    flag), ``seq_diff`` (rows whose voxel sequence differs), ``worst`` (largest
    chord difference on rows with the same sequence), ``rows``.
    """
    gidx = np.asarray(gidx)
    glen = np.asarray(glen, dtype=np.float64)
    gnnz = np.asarray(gnnz).astype(np.int64)
    m, W = gidx.shape
    if m and gnnz.max() > W:
        raise ValueError("a GPU row has %d entries, more than the %d fetched" % (gnnz.max(), W))
    cols = np.arange(W)
    no = np.diff(rowptr)
    k = np.minimum(gnnz, W)
    keep = cols[None, :] < k[:, None]
    same_n = (no == gnnz) & (gnnz <= W)
    base = rowptr[:-1]
    pos = np.clip(base[:, None] + cols[None, :], 0, max(j.size - 1, 0))
    valid = keep & same_n[:, None]
    jj = np.where(valid, j[pos] if j.size else -1, -1)
    ll = np.where(valid, ln[pos] if ln.size else 0.0, 0.0)
    eq = same_n & np.all(~keep | (gidx == jj), axis=1)
    d = np.where(valid & eq[:, None], np.abs(glen - ll), 0.0)
    flagged = near_face(margin, cond)
    wrong = (d > chord_tol(cond)[:, None]).any(axis=1) | ~eq
    unexcused = wrong & ~flagged
    vox = [gidx[d > CHORD_TOL_MM]]
    for r in np.nonzero(~eq)[0]:
        gj, gl = gidx[r, :k[r]], glen[r, :k[r]]
        oj, ol = j[rowptr[r]:rowptr[r + 1]], ln[rowptr[r]:rowptr[r + 1]]
        u = np.union1d(gj, oj)
        sg = np.zeros(u.size)
        so = np.zeros(u.size)
        np.add.at(sg, np.searchsorted(u, gj), gl)
        np.add.at(so, np.searchsorted(u, oj), ol)
        vox.append(u[np.abs(sg - so) > CHORD_TOL_MM])
    return {"chord_vox": np.concatenate(vox).astype(np.int64), "unexcused": np.nonzero(unexcused)[0],
            "seq_diff": int((~eq).sum()), "worst": float(d.max()) if d.size else 0.0, "rows": m}


class Exclusion:
    """Voxels excluded from an RSP comparison, accumulated over row chunks.

    Feed consecutive chunks of rows (GPU padded rows and the oracle's CSR rows
    of the same protons) in proton order with ``add``; chunks may start and end
    anywhere, DROP blocks of ``block`` rows are closed as they complete.  Call
    ``finish`` after the last chunk.  With ``x`` (the iterate of a single block
    step) and ``b`` the residual part (c) is applied as well.
    """

    def __init__(self, n_vox: int, block: int, x=None, b=None):
        self.n_vox = int(n_vox)
        self.block = int(block)
        self.count = np.zeros(self.n_vox, dtype=bool)
        self.chord = np.zeros(self.n_vox, dtype=bool)
        self.resid = np.zeros(self.n_vox, dtype=bool)
        self.rows_resid = 0
        # part (c): the iterate the block step starts from and the rows'
        # measurements (indexed by row, from the first row fed)
        self.x = None if x is None else np.asarray(x, dtype=np.float64).reshape(-1)
        self.b = None if b is None else np.asarray(b, dtype=np.float64).reshape(-1)
        if (self.x is None) != (self.b is None):
            raise ValueError("the residual part needs both x and b")
        self.unexcused = []
        self.seq_diff = 0
        self.rows = 0
        self.worst = 0.0
        self._blk = -1
        self._cg = np.zeros(self.n_vox, dtype=np.int64)
        self._co = np.zeros(self.n_vox, dtype=np.int64)

    def _close(self):
        if self._blk >= 0:
            self.count |= self._cg != self._co
            self._cg[:] = 0
            self._co[:] = 0

    def add(self, first_row, gidx, glen, gnnz, rowptr, j, ln, margin, cond):
        gidx = np.asarray(gidx)
        gnnz = np.asarray(gnnz).astype(np.int64)
        m, W = gidx.shape
        r = compare_row_chunk(gidx, glen, gnnz, rowptr, j, ln, margin, cond)
        self.chord[r["chord_vox"]] = True
        self.unexcused.extend((first_row + r["unexcused"]).tolist())
        self.seq_diff += r["seq_diff"]
        self.rows += m
        self.worst = max(self.worst, r["worst"])
        blk = (first_row + np.arange(m)) // self.block
        k = np.minimum(gnnz, W)
        keep = np.arange(W)[None, :] < k[:, None]
        g_rows = np.broadcast_to(np.arange(m)[:, None], (m, W))[keep]
        g_j = gidx[keep].astype(np.int64)
        o_rows = np.repeat(np.arange(m), np.diff(rowptr))
        if self.x is not None:
            self._residual(first_row, gidx, glen, keep, g_rows, rowptr, j, ln, o_rows)
        key = np.unique(o_rows.astype(np.int64) * self.n_vox + j.astype(np.int64))
        ko_rows, ko_j = key // self.n_vox, key % self.n_vox
        for b in np.unique(blk):
            if b != self._blk:
                self._close()
                self._blk = int(b)
            sel = blk == b
            rows_b = np.nonzero(sel)[0]
            lo, hi = rows_b[0], rows_b[-1] + 1
            gm = (g_rows >= lo) & (g_rows < hi)
            self._cg += np.bincount(g_j[gm], minlength=self.n_vox)
            om = (ko_rows >= lo) & (ko_rows < hi)
            self._co += np.bincount(ko_j[om], minlength=self.n_vox)

    def _residual(self, first_row, gidx, glen, keep, g_rows, rowptr, j, ln, o_rows):
        m = gidx.shape[0]
        x = self.x
        b = self.b[first_row:first_row + m]
        g_j = gidx[keep].astype(np.int64)
        g_l = np.asarray(glen, dtype=np.float64)[keep]
        o_j = np.asarray(j).astype(np.int64)
        o_l = np.asarray(ln, dtype=np.float64)

        def resid(rows, jj, ll):
            s = np.bincount(rows, weights=ll * x[jj], minlength=m)
            q = np.bincount(rows, weights=ll * ll, minlength=m)
            return np.where(q > 0, (b - s) / np.where(q > 0, q, 1.0), 0.0)

        dr = np.abs(resid(g_rows, g_j, g_l) - resid(o_rows, o_j, o_l))
        hit_g = g_l * dr[g_rows] > RESID_TOL * np.abs(x[g_j])
        hit_o = o_l * dr[o_rows] > RESID_TOL * np.abs(x[o_j])
        self.resid[g_j[hit_g]] = True
        self.resid[o_j[hit_o]] = True
        self.rows_resid += int(np.union1d(g_rows[hit_g], o_rows[hit_o]).size)

    def finish(self):
        self._close()
        self._blk = -1
        return self

    @property
    def mask(self):
        return self.count | self.chord | self.resid


def solve_parity(xg, xo, hull, excluded):
    """RSP agreement over hull voxels: dict with the max relative error on the
    voxels the rule keeps (``clean_max``), its mean, the number excluded by
    count and by chord, and the max / fraction within 1e-3 over all hull
    voxels."""
    hm = np.asarray(hull).astype(bool)
    xg = np.asarray(xg, dtype=np.float64)
    xo = np.asarray(xo, dtype=np.float64)
    rel = np.abs(xg - xo) / np.maximum(np.abs(xo), 1e-30)
    ex = excluded.mask if isinstance(excluded, Exclusion) else np.asarray(excluded, dtype=bool)
    clean = hm & ~ex
    out = {"clean_max": float(rel[clean].max()) if clean.any() else 0.0,
           "clean_mean": float(rel[clean].mean()) if clean.any() else 0.0,
           "excluded": int((hm & ex).sum()),
           "all_max": float(rel[hm].max()) if hm.any() else 0.0,
           "all_mean": float(rel[hm].mean()) if hm.any() else 0.0,
           "frac_within_1e-3": float((rel[hm] <= 1e-3).mean()) if hm.any() else 1.0,
           "hull_voxels": int(hm.sum())}
    if isinstance(excluded, Exclusion):
        out["excluded_count"] = int((hm & excluded.count).sum())
        out["excluded_chord_only"] = int((hm & excluded.chord & ~excluded.count).sum())
        if excluded.x is not None:
            out["excluded_resid_only"] = int((hm & excluded.resid & ~excluded.count & ~excluded.chord).sum())
            out["rows_resid"] = excluded.rows_resid
        out["rows"] = excluded.rows
        out["rows_seq_diff"] = excluded.seq_diff
        out["rows_unexcused"] = len(excluded.unexcused)
    return out
