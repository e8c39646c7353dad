"""Algorithm 1 (image regions, Sec. III) on the GPU vs the FP64 oracle (oracle/regions.py).

Each region solves DROP with the protons that enter and exit within its
extended slices, on rows restricted to those slices; the volume takes each
region's core slices.  Checked through the C ABI: the protons per region
against the oracle's (a proton whose hull entry or exit lies within 1e-4 mm of
an interior face of a region's slices may be counted on either side), one DROP
step per region against the oracle's within 1e-3 on the voxels the comparison
rule keeps, and 6 iterations with the same free-running bounds as the
single-region solve.
"""
import numpy as np
import pytest
import torch

import oracle as O
import synth
from oracle import regions as G
from oracle.compare import Exclusion
from tests import parity_util as U

pytestmark = pytest.mark.gpu

NEAR_MM = 1e-4


@pytest.fixture(scope="module")
def tiny(cuda_device):
    cfg, rsp, hull, hist = U.scan("tiny")
    geo, rowptr, j, ln, margin, A, cond = U.oracle_rows("tiny")
    valid, s_in, s_out = G.entry_exit_slices(geo, hist)
    st, _, _ = O.prepare(geo, hist)
    ctx = U.context(cfg, hull, hist)
    yield dict(cfg=cfg, hull=hull, hist=hist, geo=geo, rows=(rowptr, j, ln), margin=margin, cond=cond,
               valid=valid, s_in=s_in, s_out=s_out, st=st, ctx=ctx)
    ctx.close()


def _near_boundary(t, e, f):
    """Protons whose hull entry or exit z lies within NEAR_MM of slice face e or
    f, where that face is inside the grid (the outer faces are not ambiguous:
    a point on them counts in the first or last slice)."""
    geo = t["geo"]
    oz, dz, nz = geo.origin[2], geo.voxel[2], geo.shape[2]
    out = np.zeros(t["valid"].size, bool)
    for col in (4, 8):
        z = t["st"][:, col]
        for face in (e, f):
            if 0 < face < nz:
                out |= np.abs(z - (oz + face * dz)) < NEAR_MM
    return out & t["valid"]


def _restrict_padded(gidx, glen, gnnz, lo_j, hi_j):
    """GPU rows keeping the entries with voxel index in [lo_j, hi_j), re-indexed."""
    W = gidx.shape[1]
    keep = (np.arange(W)[None, :] < gnnz[:, None]) & (gidx >= lo_j) & (gidx < hi_j)
    order = np.argsort(~keep, axis=1, kind="stable")
    gi = np.take_along_axis(gidx, order, axis=1) - lo_j
    gl = np.take_along_axis(glen, order, axis=1)
    return gi, gl, keep.sum(axis=1)


def _region_exclusion(t, members, e, f, block):
    """Exclusion for one region: the GPU's rows of its (oracle) members, restricted
    to its slab, against the oracle's restricted rows; the voxels of protons
    near the region's boundary faces are excluded too."""
    cfg, ctx = t["cfg"], t["ctx"]
    plane = cfg.shape[0] * cfg.shape[1]
    rowptr, j, ln = t["rows"]
    rp, jr, lr = G.restrict_rows(rowptr, j, ln, members, plane, e, f)
    idx = np.flatnonzero(members)
    gidx, glen, gnnz = ctx.rows(0, ctx.n, max_nnz=256)
    gidx, glen, gnnz = gidx.cpu().numpy()[idx], glen.cpu().numpy()[idx], gnnz.cpu().numpy()[idx]
    assert gnnz.max() <= 256
    gi, gl, gn = _restrict_padded(gidx, glen, gnnz, e * plane, f * plane)
    ex = Exclusion((f - e) * plane, block)
    ex.add(0, gi, gl, gn, rp, jr, lr, t["margin"][idx], t["cond"][idx])
    ex.finish()
    near = _near_boundary(t, e, f)
    for i in np.flatnonzero(near):
        a, b = rowptr[i], rowptr[i + 1]
        jj = j[a:b]
        jj = jj[(jj >= e * plane) & (jj < f * plane)] - e * plane
        ex.chord[jj] = True
    return ex


def _check_counts(t, counts, regions):
    for (lo, hi, e, f), c in zip(regions, counts):
        m = G.members(t["valid"], t["s_in"], t["s_out"], e, f)
        near = _near_boundary(t, e, f)
        assert abs(c - int(m.sum())) <= int(near.sum()), (c, int(m.sum()), int(near.sum()))


@pytest.mark.parametrize("n_regions,halo", [(2, 2), (3, 1)])
def test_one_step_per_region_matches_oracle(tiny, n_regions, halo):
    t = tiny
    cfg, ctx, hull = t["cfg"], t["ctx"], t["hull"]
    x0 = hull.astype(np.float32)
    regs = G.regions(cfg.shape[2], n_regions, halo)
    B = cfg.n_protons            # one DROP block per region
    x = torch.from_numpy(x0).cuda()
    counts = ctx.solve_regions(x, n_regions, halo, 1, 0.5, B)
    ctx.synchronize()
    _check_counts(t, counts, regs)
    xo, ocounts = G.solve(t["geo"], t["hist"], n_regions, halo, 1, 0.5, B, x0.astype(np.float64), rows=t["rows"])
    xg = x.cpu().numpy().astype(np.float64)
    plane = cfg.shape[0] * cfg.shape[1]
    worst = 0.0
    for lo, hi, e, f in regs:
        m = G.members(t["valid"], t["s_in"], t["s_out"], e, f)
        ex = _region_exclusion(t, m, e, f, B)
        assert not ex.unexcused, ex.unexcused[:10]
        # this region's core slices, in its slab's voxel numbering
        core = slice((lo - e) * plane, (hi - e) * plane)
        sl = slice(lo * plane, hi * plane)
        r = U.solve_parity(xg[sl], xo[sl], hull[sl], ex.mask[core])
        worst = max(worst, r["clean_max"])
        assert r["excluded"] <= 0.01 * max(hull[sl].sum(), 1)
    print("%d regions, halo %d: counts %s (oracle %s); one step clean max %.3g"
          % (n_regions, halo, counts, ocounts, worst))
    assert worst <= 1e-3
    assert np.array_equal(xg[~hull.astype(bool)], x0[~hull.astype(bool)].astype(np.float64))


def test_six_iterations_free_running(tiny):
    t = tiny
    cfg, ctx, hull = t["cfg"], t["ctx"], t["hull"]
    x0 = hull.astype(np.float32)
    x = torch.from_numpy(x0).cuda()
    counts = ctx.solve_regions(x, 2, 2, cfg.iters, 0.5, cfg.block)
    ctx.synchronize()
    xo, ocounts = G.solve(t["geo"], t["hist"], 2, 2, cfg.iters, 0.5, cfg.block, x0.astype(np.float64),
                          rows=t["rows"])
    hm = hull.astype(bool)
    xg = x.cpu().numpy().astype(np.float64)
    rel = np.abs(xg - xo)[hm] / np.abs(xo)[hm]
    print("2 regions, 6 iterations: counts %s (oracle %s); max rel %.3g, mean %.3g, within 1e-3 %.5f"
          % (counts, ocounts, rel.max(), rel.mean(), (rel <= 1e-3).mean()))
    assert (rel <= 1e-3).mean() >= 0.999 and rel.mean() <= 1e-4


def test_one_region_is_the_solve_over_protons_with_a_hull_path(tiny):
    t = tiny
    cfg, hull = t["cfg"], t["hull"]
    import paper_1802_01070_b300 as pct
    x0 = torch.from_numpy(hull.astype(np.float32)).cuda()
    xr = x0.clone()
    counts = t["ctx"].solve_regions(xr, 1, 0, 2, 0.5, 3200)
    keep = np.flatnonzero(t["valid"])
    assert abs(counts[0] - keep.size) <= int(_near_boundary(t, 0, cfg.shape[2]).sum())
    with pct.Context(cfg.shape, cfg.voxel, cfg.origin, hull=hull) as c2:
        st = t["ctx"].hull_states().cpu().numpy()
        gk = np.flatnonzero(st[:, 10] > 0.5)
        c2.load_histories({k: torch.from_numpy(np.ascontiguousarray(v[gk])).cuda() for k, v in t["hist"].items()})
        xs = x0.clone()
        c2.solve(xs, 2, 0.5, 3200)
        c2.synchronize()
    hm = hull.astype(bool)
    d = (torch.abs(xr - xs)[torch.from_numpy(hm).cuda()] / xs[torch.from_numpy(hm).cuda()]).max().item()
    assert d <= 1e-4, d
    with pytest.raises(pct.PctError) as e:
        t["ctx"].solve_regions(xr, 0, 0, 1, 0.5, 3200)
    assert e.value.status == pct.PCT_ERR_ARG
