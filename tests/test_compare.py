"""The comparison rule of oracle.compare on hand-made rows (CPU).

Checks that identical rows exclude nothing, that a chord difference beyond
tolerance excludes its voxel only on an oracle-flagged (near-face) row and is
reported as an unexcused disagreement otherwise, that the tolerance grows with
the row's crossing conditioning, that DROP counts are compared per block, and
that a row whose residual moved excludes its voxels in a single block step.
"""
import numpy as np

from oracle.compare import (NEAR_FACE_MM, RESID_TOL, Exclusion, chord_tol, compare_row_chunk, near_face,
                            solve_parity)


def _rows():
    # oracle CSR rows of 3 protons over a 10-voxel grid
    rowptr = np.array([0, 3, 5, 8])
    j = np.array([1, 2, 3, 4, 5, 3, 6, 7], dtype=np.int32)
    ln = np.array([1.0, 0.5, 0.7, 1.2, 0.3, 0.9, 1.1, 0.2])
    return rowptr, j, ln


def _pad(rowptr, j, ln, W=4):
    m = rowptr.size - 1
    gi = np.zeros((m, W), np.int32)
    gl = np.zeros((m, W), np.float32)
    nnz = np.diff(rowptr).astype(np.int32)
    for i in range(m):
        a, b = rowptr[i], rowptr[i + 1]
        gi[i, :b - a] = j[a:b]
        gl[i, :b - a] = ln[a:b]
    return gi, gl, nnz


def test_identical_rows_exclude_nothing():
    rowptr, j, ln = _rows()
    gi, gl, nnz = _pad(rowptr, j, ln)
    margin, cond = np.ones(3), np.ones(3)
    r = compare_row_chunk(gi, gl, nnz, rowptr, j, ln, margin, cond)
    assert r["chord_vox"].size == 0 and r["unexcused"].size == 0 and r["seq_diff"] == 0
    ex = Exclusion(10, 2)
    ex.add(0, gi, gl, nnz, rowptr, j, ln, margin, cond)
    ex.finish()
    assert not ex.mask.any()


def test_chord_difference_excludes_its_voxel_and_fails_unflagged_rows():
    rowptr, j, ln = _rows()
    gi, gl, nnz = _pad(rowptr, j, ln)
    gl[1, 1] += 0.01                     # voxel 5 of row 1 off by 1e-2 mm
    margin, cond = np.ones(3), np.ones(3)
    r = compare_row_chunk(gi, gl, nnz, rowptr, j, ln, margin, cond)
    assert r["unexcused"].tolist() == [1] and r["chord_vox"].tolist() == [5]
    margin[1] = 0.5 * NEAR_FACE_MM       # a near-face row: excused, voxel still excluded
    r = compare_row_chunk(gi, gl, nnz, rowptr, j, ln, margin, cond)
    assert r["unexcused"].size == 0 and r["chord_vox"].tolist() == [5]
    # a badly conditioned crossing: the row is correct within its tolerance,
    # but the voxel's DROP input differs, so the voxel is still excluded
    margin[1] = 1.0
    cond[1] = 2000.0
    assert chord_tol(2000.0) > 0.01
    r = compare_row_chunk(gi, gl, nnz, rowptr, j, ln, margin, cond)
    assert r["unexcused"].size == 0 and r["chord_vox"].tolist() == [5]
    # the near-face window widens with the conditioning
    assert not near_face(2 * NEAR_FACE_MM, 1.0) and near_face(2 * NEAR_FACE_MM, 1000.0)
    # below the flat chord tolerance nothing is excluded
    gl[1, 1] = ln[4] + 0.001
    r = compare_row_chunk(gi, gl, nnz, rowptr, j, ln, np.ones(3), np.ones(3))
    assert r["unexcused"].size == 0 and r["chord_vox"].size == 0


def test_sequence_difference_and_block_counts():
    rowptr, j, ln = _rows()
    gi, gl, nnz = _pad(rowptr, j, ln)
    # row 2 on the GPU resolves a grazing crossing into voxel 8 as well
    gi[2, 3], gl[2, 3] = 8, 0.004
    nnz[2] = 4
    margin, cond = np.ones(3), np.ones(3)
    r = compare_row_chunk(gi, gl, nnz, rowptr, j, ln, margin, cond)
    assert r["unexcused"].tolist() == [2] and r["seq_diff"] == 1
    margin[2] = 0.0
    ex = Exclusion(10, 2)                # blocks {0, 1}, {2}
    ex.add(0, gi[:2], gl[:2], nnz[:2], rowptr[:3], j[:5], ln[:5], margin[:2], cond[:2])
    ex.add(2, gi[2:], gl[2:], nnz[2:], rowptr[2:] - rowptr[2], j[5:], ln[5:], margin[2:], cond[2:])
    ex.finish()
    assert np.nonzero(ex.count)[0].tolist() == [8] and np.nonzero(ex.chord)[0].tolist() == [8]
    assert ex.unexcused == [] and ex.rows == 3
    xo = np.ones(10)
    xg = np.ones(10)
    xg[8] = 1.5
    hull = np.ones(10, bool)
    p = solve_parity(xg, xo, hull, ex)
    assert p["clean_max"] == 0.0 and p["excluded"] == 1 and p["all_max"] == 0.5


def test_residual_part_excludes_the_voxels_of_a_row_whose_residual_moved():
    # row 0 of the oracle: voxels 1, 2, 3; on the GPU its hull entry moved along
    # a grazing tracker line, so the first chord is 0.5 mm shorter while the far
    # chords agree exactly.  Its residual r_0 = (b - a.x) / ||a||^2 differs, and
    # with it the update of voxels 2 and 3, where nothing else differs.
    rowptr, j, ln = _rows()
    gi, gl, nnz = _pad(rowptr, j, ln)
    gl[0, 0] -= 0.5
    margin, cond = np.zeros(3), np.ones(3)     # flagged: the row differs legitimately
    x = np.ones(10)
    b = np.array([2.5, 1.5, 2.2])
    ex = Exclusion(10, 3)
    ex.add(0, gi, gl, nnz, rowptr, j, ln, margin, cond)
    ex.finish()
    assert np.nonzero(ex.mask)[0].tolist() == [1]           # by chord only
    exr = Exclusion(10, 3, x=x, b=b)
    exr.add(0, gi, gl, nnz, rowptr, j, ln, margin, cond)
    exr.finish()
    assert np.nonzero(exr.mask)[0].tolist() == [1, 2, 3] and exr.rows_resid == 1
    # by hand: r = (2.5 - 2.2) / 1.74 on the oracle's row, (2.5 - 1.7) / 0.74 on
    # the GPU's; a chord of 0.5 mm times that difference is far above RESID_TOL
    r_o = (2.5 - 2.2) / (1.0 + 0.25 + 0.49)
    r_g = (2.5 - 1.7) / (0.25 + 0.25 + 0.49)
    assert 0.5 * abs(r_g - r_o) > RESID_TOL
    # a compensating chord shift between two voxels of equal x leaves r unchanged:
    # only the chord part excludes them
    gi, gl, nnz = _pad(rowptr, j, ln)
    gl[1, 0] += 0.01
    gl[1, 1] -= 0.01
    exr = Exclusion(10, 3, x=x, b=b)
    exr.add(0, gi, gl, nnz, rowptr, j, ln, margin, cond)
    exr.finish()
    assert exr.rows_resid == 0 and np.nonzero(exr.mask)[0].tolist() == [4, 5]


def test_residual_part_is_relative_to_the_voxel_value():
    # a small residual change: below RESID_TOL x_j where x_j = 1, above it on a
    # voxel whose value is 0.01 (the RSP tolerance is relative)
    rowptr, j, ln = _rows()
    gi, gl, nnz = _pad(rowptr, j, ln)
    gl[2, 2] += 1e-4                     # row 2: voxels 3, 6, 7; the last chord 1e-4 mm longer
    margin, cond = np.zeros(3), np.ones(3)
    b = np.array([2.2, 1.5, 3.0])
    x = np.ones(10)
    r_o = (3.0 - 2.2) / (0.81 + 1.21 + 0.04)
    r_g = (3.0 - 2.2 - 1e-4) / (0.81 + 1.21 + (0.2 + 1e-4) ** 2)
    dr = abs(r_g - r_o)
    assert 1.1 * dr < RESID_TOL * 1.0      # the longest chord on a voxel of value 1: kept
    assert 0.9 * dr > RESID_TOL * 0.01     # the 0.9 mm chord on a voxel of value 0.01: left out
    ex = Exclusion(10, 3, x=x, b=b)
    ex.add(0, gi, gl, nnz, rowptr, j, ln, margin, cond)
    ex.finish()
    assert not ex.resid.any()
    x[3] = 0.01
    b2 = b.copy()
    b2[2] = 3.0 - 0.9 + 0.009            # keep the residual the same size with x_3 = 0.01
    ex = Exclusion(10, 3, x=x, b=b2)
    ex.add(0, gi, gl, nnz, rowptr, j, ln, margin, cond)
    ex.finish()
    assert np.nonzero(ex.resid)[0].tolist() == [3]
