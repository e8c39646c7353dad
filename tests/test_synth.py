"""Seeded synthetic scans: shapes, determinism and the beam model's statistics."""
import math

import numpy as np
import pytest
import torch

import synth


def test_phantom_shapes_and_hull():
    for name in ("tiny", "diff"):
        cfg = synth.CONFIGS[name]
        rsp, hull = synth.phantom(cfg)
        assert rsp.shape == (cfg.n_vox,) and hull.shape == (cfg.n_vox,)
        assert hull.dtype == torch.uint8
        assert torch.all((rsp > 0) == (hull > 0))
    rsp, _ = synth.phantom(synth.CONFIGS["tiny"])
    assert np.allclose(np.unique(rsp.numpy()), [0.0, 0.3, 1.0, 1.1, 1.6])


def test_histories_are_seeded_and_shaped_like_the_scan():
    cfg = synth.scaled(synth.CONFIGS["tiny"], 4000)
    a = synth.histories(cfg, "cpu")
    b = synth.histories(cfg, "cpu")
    for k in synth.HIST_FIELDS:
        assert a[k].dtype == torch.float32 and a[k].shape == (4000,)
        assert torch.equal(a[k], b[k])
    U = synth.tracker_half_span(cfg)
    c, s = torch.cos(a["phi"]), torch.sin(a["phi"])
    u_in = a["in_x"] * c + a["in_y"] * s
    u_out = a["out_x"] * c + a["out_y"] * s
    assert torch.allclose(u_in, torch.full_like(u_in, -U), atol=1e-3)
    assert torch.allclose(u_out, torch.full_like(u_out, U), atol=1e-3)
    # 90 angles in 4-degree steps, about equally used
    k = torch.round(a["phi"] / (2 * math.pi / 90)).long()
    counts = torch.bincount(k, minlength=90)
    assert counts.numel() == 90 and counts.min() >= 4000 // 90 - 1
    assert abs(a["theta_in"].std().item() - 5e-3) < 5e-4
    assert (a["wepl"] >= 0).float().mean() > 0.99
    assert a["wepl"].max().item() < 1.7 * 2 * 28.0 + 5
