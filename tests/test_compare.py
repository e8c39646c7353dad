"""The comparison rule of oracle.compare on hand-made rows (CPU).

Checks that identical rows exclude nothing, that a chord difference beyond
tolerance excludes its voxel only on an oracle-flagged (near-face) row and is
reported as an unexcused disagreement otherwise, that the tolerance grows with
the row's crossing conditioning, and that DROP counts are compared per block.
"""
import numpy as np

from oracle.compare import NEAR_FACE_MM, Exclusion, chord_tol, compare_row_chunk, near_face, solve_parity


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
