"""Full-size workloads on the GPU, checked where the oracle can follow.

At the sizes the benchmarks run (torso 1.16e8 protons, head 1e7, large
2.61e8), in the benchmark's launch configuration, the oracle cannot build all
rows, so it checks what it can compute one by one -- MLP points and rows of
sampled protons, one DROP block of 320000 protons -- and a property that holds
at any size, the adjoint identity <A x, y> = <x, A^T y> over every proton.
"""
import numpy as np
import pytest
import torch

import oracle as O
import paper_1802_01070_b300 as pct
import synth
from tests import parity_util as U

pytestmark = pytest.mark.gpu


def _full(name):
    cfg = synth.CONFIGS[name]
    rsp, hull = synth.phantom(cfg)
    hist = synth.histories(cfg, "cuda", chunk=1 << 24, rsp=rsp)
    ctx = pct.Context(cfg.shape, cfg.voxel, cfg.origin, hull=hull.numpy())
    ctx.load_histories(hist)
    return cfg, rsp.numpy(), hull.numpy(), hist, ctx


def _sampled_rows(cfg, hull, hist, ctx, n_ranges=16, width=128, seed=0):
    rng = np.random.default_rng(seed)
    geo = U.geometry(cfg, hull)
    excused = rows = 0
    worst_pt = 0.0
    for a in rng.integers(0, cfg.n_protons - width, n_ranges):
        a = int(a)
        sub = {k: v[a:a + width].cpu().numpy() for k, v in hist.items()}
        rowptr, j, ln, margin, cond = O.rows(geo, sub, with_cond=True)
        st = ctx.hull_states(a, width).cpu().numpy().astype(np.float64)
        ost, _, _ = O.prepare(geo, sub)
        dL = np.abs((st[:, 1] - st[:, 0]) - (ost[:, 1] - ost[:, 0]))
        gidx, glen, gnnz = ctx.rows(a, width, max_nnz=1024)
        n, ex, worst, bad = U.compare_rows(gidx.cpu().numpy(), glen.cpu().numpy().astype(np.float64),
                                           gnnz.cpu().numpy(), rowptr, j, ln, margin, cond=cond, dL=dL)
        assert not bad, bad[:5]
        rows += n
        excused += ex
        pts, npts = ctx.mlp(a, width, max_pts=1024)
        opts, onpts = O.mlp_points(geo, sub, 1024)
        pts, npts = pts.cpu().numpy(), npts.cpu().numpy()
        for i in range(width):
            if npts[i] == onpts[i]:
                if npts[i] > 0:
                    worst_pt = max(worst_pt, float(np.abs(pts[i, :npts[i]] - opts[i, :npts[i]]).max()))
            else:
                assert margin[i] < U.NEAR_FACE_MM
    assert worst_pt <= U.MLP_TOL_MM
    assert excused <= 0.02 * rows
    return rows, excused, worst_pt


def _adjoint_identity(ctx, cfg, seed=1):
    g = torch.Generator(device="cuda").manual_seed(seed)
    x = torch.rand(cfg.n_vox, generator=g, device="cuda") + 0.2
    y = torch.randn(ctx.n, generator=g, device="cuda")
    ax = ctx.forward(x)
    aty = ctx.adjoint(y)
    lhs = float((ax.double() * y.double()).sum())
    rhs = float((x.double() * aty.double()).sum())
    scale = float((ax.double().abs() * y.double().abs()).sum())
    assert abs(lhs - rhs) <= 1e-5 * scale, (lhs, rhs, scale)


def test_torso_full_size():
    cfg, rsp, hull, hist, ctx = _full("torso")
    rows, excused, worst = _sampled_rows(cfg, hull, hist, ctx)
    print("torso: %d sampled rows, %d near-face, MLP worst %.3g mm" % (rows, excused, worst))
    _adjoint_identity(ctx, cfg)
    # one DROP block in the benchmark's launch shape (block 320000, fused, 256 threads)
    B = cfg.block
    sub = {k: v[:B].clone() for k, v in hist.items()}
    ctx.close()
    del hist
    torch.cuda.empty_cache()
    with pct.Context(cfg.shape, cfg.voxel, cfg.origin, hull=hull) as c1:
        c1.load_histories(sub)
        x = torch.from_numpy(hull.astype(np.float32)).cuda()
        c1.solve(x, 1, cfg.lam, B)
        c1.synchronize()
        gidx, glen, gnnz = c1.rows(0, B, max_nnz=1024)
        gidx, glen, gnnz = gidx.cpu().numpy(), glen.cpu().numpy().astype(np.float64), gnnz.cpu().numpy()
    sub_np = {k: v.cpu().numpy() for k, v in sub.items()}
    geo = U.geometry(cfg, hull)
    rowptr, j, ln, margin = O.rows(geo, sub_np)
    A = O.csr(rowptr, j, ln, geo.n_vox)
    xo = O.drop(A, sub_np["wepl"].astype(np.float64), 1, cfg.lam, B, hull.astype(np.float64))
    # voxels whose DROP count differs, or that a row crosses with a chord that
    # FP32 and FP64 resolve differently (grazing crossing), are counted apart
    diff = U.structure_diff_voxels(gidx, gnnz, rowptr, j, B, geo.n_vox)
    diff |= U.chord_diff_voxels(gidx, glen, gnnz, rowptr, j, ln, geo.n_vox)
    clean_max, n_diff, all_max, frac = U.solve_parity(x.cpu().numpy().astype(np.float64), xo, hull, diff)
    print("torso block of %d: clean max rel %.3g, %d structure- or chord-differing voxels, all max "
          "%.3g, %.5f within 1e-3" % (B, clean_max, n_diff, all_max, frac))
    assert clean_max <= 1e-3 and frac >= 0.999 and n_diff <= 0.01 * hull.sum()


def test_head_full_size():
    cfg, rsp, hull, hist, ctx = _full("head")
    rows, excused, worst = _sampled_rows(cfg, hull, hist, ctx, seed=2)
    print("head: %d sampled rows, %d near-face, MLP worst %.3g mm" % (rows, excused, worst))
    _adjoint_identity(ctx, cfg, seed=3)
    # the stored CSR rows hold as many entries as the fused rows of the same protons
    ctx.set_option(pct.PCT_OPT_MODE, pct.PCT_MODE_CSR)
    ctx.build_rows()
    total = 0
    for a in range(0, ctx.n, 1 << 21):
        c = min(ctx.n, a + (1 << 21)) - a
        total += int(ctx.rows(a, c, max_nnz=0)[2].sum().item())
    assert int(ctx.stat(pct.PCT_STAT_ROW_ENTRIES)) == total
    ctx.close()


def test_large_full_size():
    cfg, rsp, hull, hist, ctx = _full("large")
    rows, excused, worst = _sampled_rows(cfg, hull, hist, ctx, n_ranges=8, seed=4)
    print("large: %d sampled rows, %d near-face, MLP worst %.3g mm" % (rows, excused, worst))
    _adjoint_identity(ctx, cfg, seed=5)
    ctx.close()
