"""Hull distance map of a context against a brute-force chessboard distance.

The hull search that starts every path (pct_create: a path starts where the
entry line first enters a hull voxel) skips empty space with a per-voxel map of
the chessboard distance to the nearest hull voxel.  A wrong distance that is too
large would let the search jump over a hull voxel, so the map is checked voxel
by voxel here; the hull entry states themselves are checked against the oracle
in test_gpu_parity.py.
"""
import numpy as np
import pytest
import torch
from scipy import ndimage

import paper_1802_01070_b300 as pct
import synth

pytestmark = pytest.mark.gpu


def _brute(mask):
    """min over hull voxels h of max(|dz|, |dy|, |dx|), capped at 255."""
    nz, ny, nx = mask.shape
    hz, hy, hx = np.nonzero(mask)
    if hz.size == 0:
        return np.full(mask.shape, 255, np.int64)
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    best = np.full(mask.shape, 1 << 30, np.int64)
    for a, b, c in zip(hz, hy, hx):
        best = np.minimum(best, np.maximum(np.maximum(np.abs(z - a), np.abs(y - b)), np.abs(x - c)))
    return np.minimum(best, 255)


def _gpu_dist(mask):
    nz, ny, nx = mask.shape
    with pct.Context((nx, ny, nz), 1.0, (-nx / 2, -ny / 2, -nz / 2), hull=mask) as ctx:
        d = ctx.hull_distance()
        torch.cuda.synchronize()
        return d.cpu().numpy().astype(np.int64)


def test_sparse_ragged_grid_matches_brute_force():
    rng = np.random.default_rng(11)
    mask = np.zeros((11, 23, 37), np.uint8)
    for _ in range(6):
        mask[rng.integers(0, 11), rng.integers(0, 23), rng.integers(0, 37)] = 1
    assert np.array_equal(_gpu_dist(mask), _brute(mask))


def test_phantom_hull_matches_chessboard_transform():
    cfg = synth.CONFIGS["tiny"]
    _, hull = synth.phantom(cfg)
    nx, ny, nz = cfg.shape
    mask = hull.numpy().astype(np.uint8).reshape(nz, ny, nx)
    ref = np.minimum(ndimage.distance_transform_cdt(1 - mask, metric="chessboard"), 255)
    assert np.array_equal(_gpu_dist(mask), ref)


def test_distance_caps_at_255():
    mask = np.zeros((3, 4, 300), np.uint8)
    mask[1, 2, 0] = 1
    d = _gpu_dist(mask)
    assert np.array_equal(d, _brute(mask))
    assert d[1, 2, 299] == 255 and d[1, 2, 254] == 254


def test_empty_and_full_hull():
    assert (_gpu_dist(np.zeros((4, 5, 6), np.uint8)) == 255).all()
    assert (_gpu_dist(np.ones((4, 5, 6), np.uint8)) == 0).all()


def test_hull_entry_on_a_non_convex_hull_matches_oracle():
    """Hull entry and exit through a hollow shell, a one-voxel wall and isolated
    voxels: the skipping search must stop at the same first hull voxel as the
    oracle's voxel-by-voxel search (thin features are where a jump too long
    would show)."""
    import oracle as O
    from tests import parity_util as U
    cfg, rsp, hull, hist = U.scan("tiny", 30000)
    nx, ny, nz = cfg.shape
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    cx, cy = x - nx / 2 + 0.5, y - ny / 2 + 0.5
    r = np.hypot(cx, cy)
    mask = ((r >= 20) & (r <= 28)) | (x == 10)
    rng = np.random.default_rng(5)
    for _ in range(40):
        mask[rng.integers(0, nz), rng.integers(0, ny), rng.integers(0, nx)] = True
    mask = mask.astype(np.uint8).reshape(-1)
    ctx = U.context(cfg, mask, hist)
    st = ctx.hull_states().cpu().numpy().astype(np.float64)
    ctx.close()
    geo = U.geometry(cfg, mask)
    ost, ovalid, omargin = O.prepare(geo, hist)
    gvalid = st[:, 10] > 0.5
    mism = np.flatnonzero(gvalid != ovalid)
    assert np.all(omargin[mism] < U.NEAR_FACE_MM), mism[:10]
    both = gvalid & ovalid
    assert both.sum() > 0.5 * len(gvalid)
    for col in (0, 1, 2, 4, 6, 8):
        d = np.abs(st[both, col] - ost[both, col])
        ok = (d <= U.MLP_TOL_MM) | (omargin[both] < U.NEAR_FACE_MM)
        assert ok.all(), (col, d.max())
