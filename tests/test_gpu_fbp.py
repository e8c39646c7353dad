"""FBP initial iterate (Sec. I) on the GPU vs the FP64 oracle (oracle/fbp.py).

The filtered sinogram must equal the oracle's to FP32 rounding of FP64 sums
(relative 1e-6 of its largest value), and the image (FP32 back-projection
over all angles) the oracle's within 1e-4 of its largest value, voxel by
voxel on the tiny scan and on sampled voxels of the full torso (1.16e8
protons).  Bin decisions are FP64 on both sides; a proton within 1e-9 mm of a
bin edge could fall on either side, and none does in these scans.
"""
import math

import numpy as np
import pytest
import torch

import paper_1802_01070_b300 as pct
import synth
from oracle import clean as C
from oracle import fbp as F

pytestmark = pytest.mark.gpu


def _near_edges(hist, bins):
    _, t, v = C.bin_coordinates(hist)
    ft = (t - bins["t_min"]) / bins["dt"]
    fv = (v - bins["v_min"]) / bins["dv"]
    return int(((np.abs(ft - np.round(ft)) * bins["dt"] < 1e-9) |
                (np.abs(fv - np.round(fv)) * bins["dv"] < 1e-9)).sum())


def _params(bins):
    return F.FbpParams(**bins)


def test_fbp_matches_oracle_tiny(cuda_device):
    cfg = synth.CONFIGS["tiny"]
    rsp, hull = synth.phantom(cfg)
    hist = synth.to_numpy(synth.histories(cfg, "cpu", rsp=rsp))
    bins = synth.fbp_bins(cfg)
    assert _near_edges(hist, bins) == 0
    with pct.Context(cfg.shape, cfg.voxel, cfg.origin, hull=hull.numpy()) as ctx:
        ctx.load_histories({k: torch.from_numpy(v).cuda() for k, v in hist.items()})
        x, q = ctx.fbp(**bins, sinogram=True)
        x, q = x.cpu().numpy().astype(np.float64), q.cpu().numpy().astype(np.float64)
    p = _params(bins)
    _, mean = F.sinogram(hist, p)
    qo = F.ramp_filter(mean, p.dt)
    assert np.max(np.abs(q - qo)) <= 1e-6 * np.max(np.abs(qo))
    xo = F.fbp(hist, p, cfg.shape, (cfg.voxel,) * 3, cfg.origin, hull=hull.numpy())
    err = np.max(np.abs(x - xo))
    print("tiny FBP: sinogram max diff %.3g, image max diff %.3g (image max %.3g)"
          % (np.max(np.abs(q - qo)), err, np.max(np.abs(xo))))
    assert err <= 1e-4 * np.max(np.abs(xo))
    hm = hull.numpy().astype(bool)
    assert np.all(x[~hm] == 0.0)
    # the image is an RSP map: water-like inside the cylinder
    assert 0.8 < np.median(x[hm]) < 1.2


def test_fbp_full_size_torso_sampled(cuda_device):
    cfg = synth.CONFIGS["torso"]
    rsp, hull = synth.phantom(cfg)
    hist = synth.histories(cfg, "cuda", chunk=1 << 24, rsp=rsp)
    bins = synth.fbp_bins(cfg)
    with pct.Context(cfg.shape, cfg.voxel, cfg.origin, hull=hull.numpy()) as ctx:
        ctx.load_histories(hist)
        x, q = ctx.fbp(**bins, sinogram=True)
        x, q = x.cpu().numpy().astype(np.float64), q.cpu().numpy().astype(np.float64)
    hn = {k: v.cpu().numpy() for k, v in hist.items()}
    del hist
    torch.cuda.empty_cache()
    p = _params(bins)
    # sinogram rows holding a proton within 1e-9 mm of a bin edge may differ
    # (the proton's bin is decided by rounding); the filter spreads a bin's
    # difference along its row, so such rows are left out of the row check
    phi, t, v = C.bin_coordinates(hn)
    ft, fv = (t - p.t_min) / p.dt, (v - p.v_min) / p.dv
    near = (np.abs(ft - np.round(ft)) * p.dt < 1e-9) | (np.abs(fv - np.round(fv)) * p.dv < 1e-9)
    a = np.floor(phi / p.angle_step + 0.5).astype(np.int64) % p.n_angle
    rows_near = set()
    for i in np.flatnonzero(near):
        for l in {int(np.floor(fv[i] - 1e-6)), int(np.floor(fv[i] + 1e-6))}:
            rows_near.add((int(a[i]), l))
    _, mean = F.sinogram(hn, p)
    del hn
    qo = F.ramp_filter(mean, p.dt)
    ok_rows = np.ones((p.n_angle, p.n_v), bool)
    for aa, l in rows_near:
        if 0 <= l < p.n_v:
            ok_rows[aa, l] = False
    dq = np.abs(q - qo)[ok_rows]
    assert dq.max() <= 1e-6 * np.max(np.abs(qo))
    rng = np.random.default_rng(4)
    hm = hull.numpy().astype(bool)
    vox = np.concatenate([rng.choice(np.flatnonzero(hm), 20000, replace=False),
                          rng.choice(np.flatnonzero(~hm), 2000, replace=False)])
    # the back-projection of the GPU's own filtered sinogram, in FP64
    xq = np.where(hm[vox], F.backproject(q, p, cfg.shape, (cfg.voxel,) * 3, cfg.origin, voxels=vox), 0.0)
    err_bp = np.max(np.abs(x[vox] - xq))
    # and of the oracle's, on the voxels no excused row reaches
    xo = np.where(hm[vox], F.backproject(qo, p, cfg.shape, (cfg.voxel,) * 3, cfg.origin, voxels=vox), 0.0)
    l_vox = (np.asarray(vox) // (cfg.shape[0] * cfg.shape[1]))
    far = np.array([all(ok_rows[:, l]) for l in l_vox])
    err = np.max(np.abs(x[vox] - xo)[far]) if far.any() else 0.0
    print("torso FBP: %d protons near a bin edge (%d sinogram rows excused); %d sampled voxels: back-"
          "projection max diff %.3g, end to end %.3g on %d voxels (image max %.3g); RSP mean abs error vs "
          "truth %.3g" % (int(near.sum()), len(rows_near), vox.size, err_bp, err, int(far.sum()),
                          np.max(np.abs(xo)), np.mean(np.abs(x[hm] - rsp.numpy()[hm]))))
    assert err_bp <= 1e-4 * np.max(np.abs(xo))
    assert err <= 1e-4 * np.max(np.abs(xo))
    assert len(rows_near) <= 0.01 * ok_rows.size


def test_fbp_edge_cases(cuda_device):
    cfg = synth.scaled(synth.CONFIGS["tiny"], 2000, name="tiny-fbp-edge")
    rsp, hull = synth.phantom(cfg)
    hist = synth.histories(cfg, "cpu", rsp=rsp)
    bins = synth.fbp_bins(cfg)
    with pct.Context(cfg.shape, cfg.voxel, cfg.origin, hull=hull.numpy()) as ctx:
        ctx.load_histories({k: v[:0].cuda() for k, v in hist.items()})
        x = ctx.fbp(**bins)
        assert torch.all(x == 0)
        ctx.load_histories({k: v.cuda() for k, v in hist.items()})
        for bad in (dict(bins, n_angle=0), dict(bins, n_angle=5000), dict(bins, dt=-1.0),
                    dict(bins, dv=float("inf"))):
            with pytest.raises(pct.PctError) as e:
                ctx.fbp(**bad)
            assert e.value.status == pct.PCT_ERR_ARG
        # v bins that miss every slice: 0 everywhere
        x = ctx.fbp(**dict(bins, v_min=1e3))
        assert torch.all(x == 0)
