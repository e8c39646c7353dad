"""Pins of the Algorithm 1 oracle (oracle/regions.py) against things other than itself.

CPU only.  The paper's own example of the regions, one region being the plain
DROP solve, regions that each cover the whole volume reproducing it, region
membership from the end points of the MLP polyline, and restricted rows that
add up to the full rows.
"""
import numpy as np
import pytest

import oracle as O
import synth
from oracle import regions as G


def test_the_papers_example_regions():
    # 20 slices, two regions: slices 0-12 and 7-19, kept 0-9 and 10-19
    assert G.regions(20, 2, 3) == [(0, 10, 0, 13), (10, 20, 7, 20)]
    assert G.regions(8, 4, 1) == [(0, 2, 0, 3), (2, 4, 1, 5), (4, 6, 3, 7), (6, 8, 5, 8)]
    assert G.regions(7, 3, 0) == [(0, 2, 0, 2), (2, 4, 2, 4), (4, 7, 4, 7)]


@pytest.fixture(scope="module")
def scan():
    cfg = synth.scaled(synth.CONFIGS["tiny"], 12000, name="tiny-regions")
    rsp, hull = synth.phantom(cfg)
    hist = synth.to_numpy(synth.histories(cfg, "cpu", rsp=rsp))
    geo = O.Geometry(cfg.shape, (cfg.voxel,) * 3, cfg.origin, mask=hull.numpy())
    rowptr, j, ln, _ = O.rows(geo, hist)
    return cfg, hull.numpy(), hist, geo, (rowptr, j, ln)


def test_one_region_is_the_plain_solve(scan):
    cfg, hull, hist, geo, rows = scan
    x0 = hull.astype(np.float64)
    x, counts = G.solve(geo, hist, 1, 0, 2, 0.5, 3200, x0, rows=rows)
    valid = G.entry_exit_slices(geo, hist)[0]
    assert counts == [int(valid.sum())]
    # the region's blocks are 3200 consecutive protons of its own list (those
    # with a hull path): the plain DROP over those protons' rows
    rowptr, j, ln = rows
    keep = np.flatnonzero(valid)
    A = O.csr(*rows, geo.n_vox)[keep]
    xo = O.drop(A, hist["wepl"].astype(np.float64)[keep], 2, 0.5, 3200, x0)
    assert np.max(np.abs(x - xo)) < 1e-12


def test_regions_covering_the_volume_reproduce_the_plain_solve(scan):
    # halo >= nz: every region's slab is the whole volume and every proton
    # with a hull path belongs to every region
    cfg, hull, hist, geo, rows = scan
    x0 = hull.astype(np.float64)
    nz = cfg.shape[2]
    x, counts = G.solve(geo, hist, 2, nz, 2, 0.5, 3200, x0, rows=rows)
    xo, _ = G.solve(geo, hist, 1, 0, 2, 0.5, 3200, x0, rows=rows)
    assert counts[0] == counts[1] and np.max(np.abs(x - xo)) < 1e-12


def test_membership_from_the_polyline_end_points(scan):
    cfg, hull, hist, geo, rows = scan
    pts, npts = O.mlp_points(geo, hist, 512)
    valid, s_in, s_out = G.entry_exit_slices(geo, hist)
    ok = npts > 0
    assert np.array_equal(ok, valid)
    idx = np.flatnonzero(ok)
    z_in = pts[idx, 0, 2]
    z_out = pts[idx, npts[idx] - 1, 2]
    dz, oz = geo.voxel[2], geo.origin[2]
    # end points on the grid's outer faces count in the first or last slice
    nz = cfg.shape[2]
    zs_in = np.clip(np.floor((z_in - oz) / dz), 0, nz - 1)
    zs_out = np.clip(np.floor((z_out - oz) / dz), 0, nz - 1)
    assert np.array_equal(zs_in.astype(int), s_in[idx]) and np.array_equal(zs_out.astype(int), s_out[idx])
    # each region holds exactly the protons whose polyline starts and ends in
    # its extended slices
    regs = G.regions(nz, 2, 1)
    ms = []
    for lo, hi, e, f in regs:
        m = G.members(valid, s_in, s_out, e, f)
        want = np.zeros_like(valid)
        want[idx] = (zs_in >= e) & (zs_in < f) & (zs_out >= e) & (zs_out < f)
        assert np.array_equal(m, want)
        ms.append(m)
    # nearly every proton with a hull path fits a region; one that starts in a
    # region's slices and ends outside them does not belong to it
    covered = ms[0] | ms[1]
    assert not (covered & ~valid).any() and covered[valid].mean() > 0.95
    e0, f0 = regs[0][2], regs[0][3]
    assert ((zs_in >= e0) & (zs_in < f0) & (zs_out >= f0)).any()


def test_restricted_rows_add_up_to_the_full_rows(scan):
    cfg, hull, hist, geo, rows = scan
    rowptr, j, ln = rows
    plane = cfg.shape[0] * cfg.shape[1]
    nz = cfg.shape[2]
    sel = np.diff(rowptr) > 0
    m = int(sel.sum())
    total = np.zeros(m)
    for lo, hi in ((0, 3), (3, 5), (5, nz)):
        rp, jr, lr = G.restrict_rows(rowptr, j, ln, sel, plane, lo, hi)
        assert np.all((jr >= 0) & (jr < (hi - lo) * plane))
        total += np.bincount(np.repeat(np.arange(m), np.diff(rp)), weights=lr, minlength=m)
    rows_sel = np.flatnonzero(sel)
    full = np.bincount(np.repeat(np.arange(m), np.diff(rowptr)[rows_sel]),
                       weights=np.concatenate([ln[rowptr[r]:rowptr[r + 1]] for r in rows_sel]), minlength=m)
    assert np.allclose(total, full, rtol=1e-12, atol=0)
