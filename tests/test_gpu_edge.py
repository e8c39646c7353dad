"""Edge cases of the GPU path through the C ABI: empty and ragged inputs,
degenerate grids, block sizes 1 and > m, anisotropic voxels, a finer MLP step,
and error statuses."""
import math

import numpy as np
import pytest
import torch

import oracle as O
import paper_1802_01070_b300 as pct
import synth
from tests import parity_util as U

pytestmark = pytest.mark.gpu


def _sub(hist, a, b):
    return {k: np.ascontiguousarray(v[a:b]) for k, v in hist.items()}


def test_errors_and_states(cuda_device):
    cfg, rsp, hull, hist = U.scan("tiny")
    ctx = pct.Context(cfg.shape, cfg.voxel, cfg.origin, hull=hull)
    x = torch.ones(cfg.n_vox, device=cuda_device)
    with pytest.raises(pct.PctError) as e:
        ctx.solve(x, 1, 0.5, 100)                  # nothing loaded yet
    assert e.value.status == pct.PCT_ERR_STATE
    ctx.load_histories({k: torch.empty(0) for k in pct.HIST_FIELDS})
    ctx.solve(x, 3, 0.5, 100)                      # zero protons: x unchanged
    ctx.synchronize()
    assert torch.all(x == 1)
    assert ctx.forward(x).numel() == 0
    with pytest.raises(pct.PctError) as e:
        pct.pct_solve(ctx.handle, 1, 0.5, 0, x)
    assert e.value.status == pct.PCT_ERR_ARG
    with pytest.raises(pct.PctError) as e:
        pct.pct_solve(ctx.handle, -1, 0.5, 10, x)
    assert e.value.status == pct.PCT_ERR_ARG
    lib = pct.load_library()
    assert lib.pct_solve(ctx.handle, 1, 0.5, 10, None) == pct.PCT_ERR_ARG
    assert lib.pct_mlp(ctx.handle, 0, 5, 16, None, None) == pct.PCT_ERR_ARG   # range beyond n
    ctx.close()


def test_sampled_launch_timing(cuda_device):
    cfg, rsp, hull, hist = U.scan("tiny")
    ctx = pct.Context(cfg.shape, cfg.voxel, cfg.origin, hull=hull)
    ctx.load_histories({k: torch.from_numpy(v).cuda() for k, v in hist.items()})
    x = torch.from_numpy(hull.astype(np.float32)).cuda()
    ctx.set_option(pct.PCT_OPT_PERSISTENT_BLOCK, 0)   # a launch per block step, each one timed
    with pytest.raises(pct.PctError) as e:
        ctx.set_option(pct.PCT_OPT_TIMING, -1)
    assert e.value.status == pct.PCT_ERR_ARG
    blocks = math.ceil(cfg.n_protons / cfg.block)
    for period in (1, 3):
        ctx.reset_stats()
        ctx.set_option(pct.PCT_OPT_TIMING, period)
        ctx.solve(x, 2, cfg.lam, cfg.block)
        launches = ctx.stat(pct.PCT_STAT_FUSED_LAUNCHES)
        assert launches == 2 * blocks
        assert ctx.stat(pct.PCT_STAT_TIMED_LAUNCHES) == math.ceil(launches / period)
        assert ctx.stat(pct.PCT_STAT_FUSED_MS) > 0
    ctx.reset_stats()
    ctx.set_option(pct.PCT_OPT_TIMING, 0)
    ctx.solve(x, 1, cfg.lam, cfg.block)
    assert ctx.stat(pct.PCT_STAT_TIMED_LAUNCHES) == 0 and ctx.stat(pct.PCT_STAT_FUSED_MS) == 0
    ctx.close()


def test_host_upload_in_chunks_matches_device_load(cuda_device):
    """Histories from (pinned) host memory are uploaded in chunks of 2^22 protons
    with each chunk's records prepared as it lands: the records and a solve
    equal those of a device-to-device load."""
    cfg = synth.scaled(synth.CONFIGS["tiny"], (1 << 22) + 12345)
    rsp, hull = synth.phantom(cfg)
    hist = synth.histories(cfg, cuda_device, rsp=rsp)
    host = {k: v.cpu().pin_memory() for k, v in hist.items()}
    hull = hull.numpy()
    x0 = torch.from_numpy(hull.astype(np.float32)).cuda()
    out = []
    for h in (hist, host):
        with pct.Context(cfg.shape, cfg.voxel, cfg.origin, hull=hull) as ctx:
            ctx.load_histories(h)
            st = ctx.hull_states().clone()
            x = x0.clone()
            ctx.solve(x, 1, cfg.lam, 320000)
            ctx.synchronize()
            out.append((st, x))
    assert torch.equal(out[0][0], out[1][0])
    assert torch.allclose(out[0][1], out[1][1], rtol=1e-5, atol=1e-6)   # FP32 atomics order


def test_records_follow_histories_and_mlp_step(cuda_device):
    """The per-proton records are kept between calls: a repeated call reuses
    them, a new MLP step or a new history load recomputes them."""
    cfg, rsp, hull, hist = U.scan("tiny")
    a, b = _sub(hist, 0, 3000), _sub(hist, 3000, 6000)
    ctx = U.context(cfg, hull, a)
    st_a = ctx.hull_states().clone()
    ctx.reset_stats()
    _, n1 = ctx.mlp(0, 100, max_pts=1024)
    launches = ctx.stat(pct.PCT_STAT_LAUNCHES)
    assert launches == 1                                  # the MLP kernel alone: records kept
    ctx.set_option(pct.PCT_OPT_MLP_STEP_UM, 500)
    _, n2 = ctx.mlp(0, 100, max_pts=1024)
    ok = n1 > 0
    assert torch.all(n2[ok] > n1[ok])                     # finer step, records recomputed
    ctx.set_option(pct.PCT_OPT_MLP_STEP_UM, 1000)
    ctx.load_histories({k: torch.from_numpy(v).cuda() for k, v in b.items()})
    st_b = ctx.hull_states()
    ref = U.context(cfg, hull, b)
    assert torch.equal(st_b, ref.hull_states())           # the new histories' records
    assert not torch.equal(st_a, st_b)
    ref.close()
    ctx.close()


def test_memory_cap_gives_oom_status(cuda_device):
    cfg, rsp, hull, hist = U.scan("tiny")
    ctx = pct.Context(cfg.shape, cfg.voxel, cfg.origin, hull=hull)
    ctx.set_option(pct.PCT_OPT_MEM_CAP_BYTES, int(ctx.stat(pct.PCT_STAT_DEVICE_BYTES)) + 4096)
    with pytest.raises(pct.PctError) as e:
        ctx.load_histories({k: torch.from_numpy(v).cuda() for k, v in hist.items()})
    assert e.value.status == pct.PCT_ERR_OOM
    ctx.set_option(pct.PCT_OPT_MEM_CAP_BYTES, 0)
    ctx.load_histories({k: torch.from_numpy(v).cuda() for k, v in hist.items()})
    ctx.close()


def test_protons_missing_the_hull_have_empty_rows(cuda_device):
    cfg, rsp, hull, hist = U.scan("tiny")
    h = _sub(hist, 0, 2000)
    for k in ("in_z", "out_z"):
        h[k] = h[k] + 50.0                          # above the grid
    ctx = U.context(cfg, hull, h)
    idx, ln, nnz = ctx.rows(max_nnz=8)
    assert int(nnz.max()) == 0
    x = torch.from_numpy(hull.astype(np.float32)).cuda()
    x0 = x.clone()
    ctx.solve(x, 2, 0.5, 64)
    ctx.synchronize()
    assert torch.equal(x, x0)
    assert torch.all(ctx.forward(x) == 0)
    ctx.close()


@pytest.mark.parametrize("n,block", [(10007, 3200), (1500, 1), (3000, 100000)])
def test_ragged_and_extreme_block_sizes(cuda_device, n, block):
    cfg, rsp, hull, hist = U.scan("tiny")
    h = _sub(hist, 0, n)
    geo = U.geometry(cfg, hull)
    rowptr, j, ln, margin = O.rows(geo, h)
    A = O.csr(rowptr, j, ln, geo.n_vox)
    ctx = U.context(cfg, hull, h)
    x0 = hull.astype(np.float32)
    x = torch.from_numpy(x0).cuda()
    iters = 1 if block == 1 else 3
    ctx.solve(x, iters, 0.5, block)
    ctx.synchronize()
    xo = O.drop(A, h["wepl"].astype(np.float64), iters, 0.5, block, x0.astype(np.float64))
    hm = hull.astype(bool)
    rel = np.abs(x.cpu().numpy() - xo)[hm] / xo[hm]
    assert rel.max() <= 1e-3, rel.max()
    ctx.close()


def _single_voxel_hist(n, rng):
    # straight-ish protons through a 1x1x1 grid of 4 mm, trackers 20 mm away
    phi = rng.uniform(0, 2 * math.pi, n)
    t = rng.uniform(-1.5, 1.5, n)
    v = rng.uniform(-1.5, 1.5, n)
    c, s = np.cos(phi), np.sin(phi)
    th_i, ps_i = rng.normal(0, 0.01, n), rng.normal(0, 0.01, n)
    th_o, ps_o = th_i + rng.normal(0, 0.005, n), ps_i + rng.normal(0, 0.005, n)
    t2 = t + 40 * th_i
    v2 = v + 40 * ps_i
    h = {"in_x": -20 * c - t * s, "in_y": -20 * s + t * c, "in_z": v,
         "out_x": 20 * c - t2 * s, "out_y": 20 * s + t2 * c, "out_z": v2,
         "theta_in": th_i, "psi_in": ps_i, "theta_out": th_o, "psi_out": ps_o,
         "phi": phi, "wepl": rng.uniform(3.0, 5.0, n)}
    return {k: np.ascontiguousarray(v, dtype=np.float32) for k, v in h.items()}


def test_single_voxel_grid(cuda_device):
    rng = np.random.default_rng(9)
    h = _single_voxel_hist(3000, rng)
    cfg = synth.ScanConfig("one", (1, 1, 1), 4.0, "tiny", 3000, 1, 2, 0.5, 256)
    hull = np.ones(1, dtype=np.uint8)
    geo = U.geometry(cfg, hull)
    rowptr, j, ln, margin = O.rows(geo, h)
    ctx = U.context(cfg, hull, h)
    gidx, glen, gnnz = ctx.rows(max_nnz=4)
    assert np.array_equal(gnnz.cpu().numpy(), np.diff(rowptr))
    m = np.diff(rowptr) > 0
    assert np.allclose(glen.cpu().numpy()[m, 0], ln, atol=U.CHORD_TOL_MM)
    A = O.csr(rowptr, j, ln, 1)
    x = torch.ones(1, device=cuda_device)
    ctx.solve(x, 2, 0.5, 256)
    ctx.synchronize()
    xo = O.drop(A, h["wepl"].astype(np.float64), 2, 0.5, 256, np.ones(1))
    assert abs(x.item() - xo[0]) <= 1e-3 * abs(xo[0])
    ctx.close()


def test_anisotropic_voxels_offset_origin_and_fine_mlp_step(cuda_device):
    base = synth.CONFIGS["tiny"]
    cfg0, rsp0, hull0, hist = U.scan("tiny")
    h = _sub(hist, 0, 4000)
    shape, voxel, origin = (40, 52, 10), (1.6, 1.25, 0.8), (-33.0, -31.5, -4.2)
    nx, ny, nz = shape
    z, y, x = np.meshgrid((np.arange(nz) + 0.5) * voxel[2] + origin[2],
                          (np.arange(ny) + 0.5) * voxel[1] + origin[1],
                          (np.arange(nx) + 0.5) * voxel[0] + origin[0], indexing="ij")
    hull = ((x * x + y * y) <= 27.0 ** 2).astype(np.uint8).reshape(-1)
    for du_um in (None, 500):
        geo = O.Geometry(shape, voxel, origin, mask=hull, du=None if du_um is None else du_um / 1000)
        rowptr, j, ln, margin, cond = O.rows(geo, h, with_cond=True)
        ctx = pct.Context(shape, voxel, origin, hull=hull)
        if du_um is not None:
            ctx.set_option(pct.PCT_OPT_MLP_STEP_UM, du_um)
        ctx.load_histories({k: torch.from_numpy(v).cuda() for k, v in h.items()})
        gidx, glen, gnnz = ctx.rows(max_nnz=256)
        rows, excused, worst, bad = U.compare_rows(gidx.cpu().numpy(),
                                                   glen.cpu().numpy().astype(np.float64),
                                                   gnnz.cpu().numpy(), rowptr, j, ln, margin,
                                                   cond=cond)
        assert not bad, bad[:5]
        assert excused <= 0.02 * rows
        ctx.close()


def test_lanes_with_more_runs_than_slots(cuda_device):
    """A lane whose range holds more runs than its 24 shared-memory slots walks
    the runs beyond them again (once for the row's dot products, once for the
    scatter).  0.25 mm voxels with a 5 mm MLP step put about 25 runs in every
    lane's segment; one DROP block step from a known iterate must still match
    the oracle's step under the comparison rule, and A x must match the
    oracle's product."""
    cfg0, rsp0, hull0, hist = U.scan("tiny")
    h = _sub(hist, 0, 3000)
    vox = 0.25
    shape = (240, 240, 32)
    origin = tuple(-0.5 * n * vox for n in shape)
    nx, ny, nz = shape
    z, y, x = np.meshgrid((np.arange(nz) + 0.5) * vox + origin[2],
                          (np.arange(ny) + 0.5) * vox + origin[1],
                          (np.arange(nx) + 0.5) * vox + origin[0], indexing="ij")
    hull = ((x * x + y * y) <= 27.0 ** 2).astype(np.uint8).reshape(-1)
    du_um = 5000
    geo = O.Geometry(shape, (vox,) * 3, origin, mask=hull, du=du_um / 1000)
    rowptr, j, ln, margin, cond = O.rows(geo, h, with_cond=True)
    A = O.csr(rowptr, j, ln, geo.n_vox)
    ctx = pct.Context(shape, (vox,) * 3, origin, hull=hull)
    try:
        ctx.set_option(pct.PCT_OPT_MLP_STEP_UM, du_um)
        ctx.load_histories({k: torch.from_numpy(v).cuda() for k, v in h.items()})
        # the workload reaches the overflow: with one segment per lane (the 5 mm
        # step exceeds a voxel diagonal) a row whose runs outnumber 24 per
        # segment has a lane beyond its slots
        _, npts = ctx.mlp(0, len(h["wepl"]), max_pts=256)
        nseg = np.maximum(npts.cpu().numpy() - 1, 1)
        nnz = np.diff(rowptr)
        assert int((nnz > 24 * nseg).sum()) >= 100
        rng = np.random.default_rng(5)
        x0 = (hull * (1.0 + 0.1 * rng.standard_normal(hull.size))).astype(np.float32)
        xg = torch.from_numpy(x0).cuda()
        yg = ctx.forward(xg).cpu().numpy().astype(np.float64)
        yo = A @ x0.astype(np.float64)
        ok = ~np.array([U.near_face(margin[i], cond[i]) for i in range(len(yo))])
        assert np.max(np.abs(yg - yo)[ok] / np.maximum(np.abs(yo[ok]), 1.0)) <= 1e-4
        n = len(h["wepl"])
        b = h["wepl"].astype(np.float64)
        ctx.solve(xg, 1, 0.5, n)
        ctx.synchronize()
        xs = xg.cpu().numpy().astype(np.float64)
        xo = O.drop(A, b, 1, 0.5, n, x0.astype(np.float64))
        ex = U.gpu_exclusion(ctx, rowptr, j, ln, margin, cond, n, x=x0.astype(np.float64), b=b)
        r = U.solve_parity(xs, xo, hull, ex)
        print(r)
        assert r["rows_unexcused"] == 0, ex.unexcused[:10]
        assert r["clean_max"] <= 1e-3
        assert r["excluded"] <= 0.02 * hull.sum()
    finally:
        ctx.close()
