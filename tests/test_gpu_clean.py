"""Data cleaning (statistical outlier removal, Sec. IV-A) on the GPU vs the FP64 oracle.

The keep decision of every proton must equal the oracle's (oracle/clean.py),
except protons within rounding of a cut (relative margin < 1e-9: the GPU's
per-bin sums are FP64 atomics in no fixed order), which are counted; the kept
protons must replace the loaded set in order, bit for bit.  At full torso size
(1.16e8 protons, 2 % planted outliers) the oracle checks the protons of two
whole angle bins: bins are independent, so their decisions are the full scan's.
"""
import math

import numpy as np
import pytest
import torch

import paper_1802_01070_b300 as pct
import synth
from oracle import clean as C

pytestmark = pytest.mark.gpu

NEAR_CUT = 1e-9


def _ctx(cfg, hull, hist):
    ctx = pct.Context(cfg.shape, cfg.voxel, cfg.origin, hull=hull)
    ctx.load_histories({k: (v if torch.is_tensor(v) else torch.from_numpy(v)).cuda() for k, v in hist.items()})
    return ctx


def _compare(keep_g, keep_o, margin):
    near = np.abs(margin) < NEAR_CUT
    diff = keep_g != keep_o
    assert not (diff & ~near).any(), np.nonzero(diff & ~near)[0][:10]
    return int(near.sum()), int(diff.sum())


def test_clean_matches_oracle_and_compacts_in_order(cuda_device):
    cfg = synth.CONFIGS["tiny"]
    rsp, hull = synth.phantom(cfg)
    hist = synth.to_numpy(synth.histories(cfg, "cpu", rsp=rsp, outlier_frac=0.02))
    bins = synth.clean_bins(cfg)
    keep_o, margin = C.clean(hist, C.CleanParams(**bins))
    with _ctx(cfg, hull.numpy(), hist) as ctx:
        n0 = ctx.n
        kept, flags = ctx.clean(**bins, keep=True)
        keep_g = flags.cpu().numpy().astype(bool)
        assert keep_g.size == n0 and kept == int(keep_g.sum()) == ctx.n
        near, diff = _compare(keep_g, keep_o, margin)
        print("tiny: kept %d of %d (oracle %d); %d near a cut, %d decided differently"
              % (kept, n0, int(keep_o.sum()), near, diff))
        planted = synth.outlier_mask(cfg, frac=0.02).numpy()
        assert (~keep_g[planted]).mean() > 0.5
        st = ctx.hull_states().cpu().numpy()
    # the cleaned set is the kept protons, in order
    sub = {k: v[keep_g] for k, v in hist.items()}
    with _ctx(cfg, hull.numpy(), sub) as ref:
        assert ref.n == kept
        assert np.array_equal(ref.hull_states().cpu().numpy(), st)


def test_clean_edge_cases(cuda_device):
    cfg = synth.scaled(synth.CONFIGS["tiny"], 5000, name="tiny-clean-edge")
    rsp, hull = synth.phantom(cfg)
    hist = synth.to_numpy(synth.histories(cfg, "cpu", rsp=rsp))
    bins = synth.clean_bins(cfg)
    with _ctx(cfg, hull.numpy(), hist) as ctx:
        # bins that no proton reaches: everything is removed, and a solve still runs
        far = dict(bins, t_min=1e4)
        assert ctx.clean(**far) == 0 and ctx.n == 0
        x = torch.from_numpy(hull.numpy().astype(np.float32)).cuda()
        ctx.solve(x, 1, 0.5, 100)
        ctx.synchronize()
        assert ctx.clean(**bins) == 0
        for bad in (dict(bins, n_t=0), dict(bins, dt=0.0), dict(bins, k_sigma=-1.0),
                    dict(bins, angle_step=float("nan"))):
            with pytest.raises(pct.PctError) as e:
                ctx.clean(**bad)
            assert e.value.status == pct.PCT_ERR_ARG
    # a generous cut keeps every binned proton; a reload restores the set
    with _ctx(cfg, hull.numpy(), hist) as ctx:
        assert ctx.clean(**dict(bins, k_sigma=1e6)) == C.clean(hist, C.CleanParams(**dict(bins, k_sigma=1e6)))[0].sum()


def test_clean_full_size_torso(cuda_device):
    cfg = synth.CONFIGS["torso"]
    rsp, hull = synth.phantom(cfg)
    hist = synth.histories(cfg, "cuda", chunk=1 << 24, rsp=rsp, outlier_frac=0.02)
    bins = synth.clean_bins(cfg)
    step = bins["angle_step"]
    a = torch.floor(hist["phi"].double() / step + 0.5).long() % bins["n_angle"]
    pick = ((a == 0) | (a == 90)).cpu().numpy()
    sub = {k: v.cpu().numpy()[pick] for k, v in hist.items()}
    with pct.Context(cfg.shape, cfg.voxel, cfg.origin, hull=hull.numpy()) as ctx:
        ctx.load_histories(hist)
        del hist
        kept, flags = ctx.clean(**bins, keep=True)
        keep_g = flags.cpu().numpy().astype(bool)
        assert kept == int(keep_g.sum()) == ctx.n
    keep_o, margin = C.clean(sub, C.CleanParams(**bins))
    near, diff = _compare(keep_g[pick], keep_o, margin)
    print("torso: kept %d of %d; %d protons of angle bins 0 and 90 checked, %d near a cut, %d decided "
          "differently" % (kept, keep_g.size, int(pick.sum()), near, diff))
    assert pick.sum() > 1e6
