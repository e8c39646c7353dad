"""pct_solve_noalloc: the DROP reconstruction for callers that cannot allocate.

Some applications give all device memory to their own pool and forbid
cudaMalloc outside it, or cannot afford the device-wide synchronization that
cudaMalloc/cudaFree can cause in the middle of a scan.  pct_solve_noalloc runs
the same kernels as pct_solve with its scratch in fixed arrays inside the
library.  This test calls it twice in a row through the C ABI and checks each
result against the context path (pct_create + pct_load_histories + pct_solve)
within the tolerance used for two GPU runs of the same kernels (only the order
of the FP32 atomics differs).  It lives in its own file, collected last, and
needs nothing from the other test files.
"""
import numpy as np
import pytest
import torch

import paper_1802_01070_b300 as pct
import synth

pytestmark = pytest.mark.gpu

ITERS, LAM, BLOCK, N = 3, 0.5, 3200, 30000


def _scan():
    cfg = synth.scaled(synth.CONFIGS["tiny"], N, name="tiny-noalloc")
    rsp, hull = synth.phantom(cfg)
    hist = synth.histories(cfg, "cpu", rsp=rsp)
    return cfg, hull.numpy(), hist


def test_noalloc_solve_matches_context_solve_on_two_calls(cuda_device):
    cfg, hull, hist = _scan()
    dev = cuda_device
    hd = {k: v.to(dev) for k, v in hist.items()}
    x0 = torch.from_numpy(hull.astype(np.float32)).to(dev)

    with pct.Context(cfg.shape, cfg.voxel, cfg.origin, hull=hull) as ctx:
        ctx.load_histories(hd)
        x_ref = x0.clone()
        ctx.solve(x_ref, ITERS, LAM, BLOCK)
        ctx.synchronize()
    ref = x_ref.cpu().numpy()
    hm = hull.astype(bool)

    hull_dev = torch.from_numpy(hull).to(dev)
    vox = (cfg.voxel,) * 3
    for call in range(2):
        x = x0.clone()
        st = pct.pct_solve_noalloc(cfg.shape, vox, cfg.origin, hull_dev, hd, ITERS, LAM, BLOCK, x)
        assert st == pct.PCT_OK, st
        got = x.cpu().numpy()
        rel = np.abs(got - ref)[hm] / np.abs(ref)[hm]
        assert rel.max() <= 1e-4, (call, rel.max())
        assert np.array_equal(got[~hm], x0.cpu().numpy()[~hm])


def test_noalloc_call_takes_no_device_memory(cuda_device):
    # after a first call (which loads the kernels it uses), a call must leave
    # the device's free memory exactly as it found it
    cfg, hull, hist = _scan()
    dev = cuda_device
    hd = {k: v.to(dev) for k, v in hist.items()}
    hull_dev = torch.from_numpy(hull).to(dev)
    vox = (cfg.voxel,) * 3
    x = torch.from_numpy(hull.astype(np.float32)).to(dev)
    assert pct.pct_solve_noalloc(cfg.shape, vox, cfg.origin, hull_dev, hd, 1, LAM, BLOCK, x) == pct.PCT_OK
    torch.cuda.synchronize(dev)
    free0, _ = torch.cuda.mem_get_info(dev)
    assert pct.pct_solve_noalloc(cfg.shape, vox, cfg.origin, hull_dev, hd, ITERS, LAM, BLOCK, x) == pct.PCT_OK
    torch.cuda.synchronize(dev)
    free1, _ = torch.cuda.mem_get_info(dev)
    assert free1 == free0, (free0, free1)


def test_noalloc_rejects_sizes_beyond_its_limits(cuda_device):
    cfg, hull, hist = _scan()
    dev = cuda_device
    hd = {k: v.to(dev) for k, v in hist.items()}
    x = torch.ones(cfg.n_vox, device=dev)
    hull_dev = torch.from_numpy(hull).to(dev)
    vox = (cfg.voxel,) * 3
    big = (1024, 1024, 2)                      # 2^21 voxels > the limit
    xb = torch.ones(1024 * 1024 * 2, device=dev)
    hb = torch.ones(1024 * 1024 * 2, dtype=torch.uint8, device=dev)
    assert pct.pct_solve_noalloc(big, vox, cfg.origin, hb, hd, 1, LAM, BLOCK, xb) == pct.PCT_ERR_ARG
    assert torch.all(xb == 1.0)
    # the binding refuses buffers shorter than the grid before calling the library
    with pytest.raises(ValueError):
        pct.pct_solve_noalloc(cfg.shape, vox, cfg.origin, hull_dev, hd, 1, LAM, BLOCK, x[:-1])
    with pytest.raises(ValueError):
        pct.pct_solve_noalloc(cfg.shape, vox, cfg.origin, hull_dev[:-1], hd, 1, LAM, BLOCK, x)
    many = {k: torch.zeros(pct.PCT_NOALLOC_MAX_PROTONS + 1, device=dev) for k in pct.HIST_FIELDS}
    assert pct.pct_solve_noalloc(cfg.shape, vox, cfg.origin, hull_dev, many, 1, LAM, BLOCK, x) == pct.PCT_ERR_ARG
    x0 = x.clone()
    assert pct.pct_solve_noalloc(cfg.shape, vox, cfg.origin, hull_dev, hd, 1, LAM, 0, x) == pct.PCT_ERR_ARG
    assert torch.equal(x, x0)
