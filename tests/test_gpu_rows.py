"""Stored row forms (CSR; packed 1-byte step codes + 16-bit chords) through the C ABI.

The stored rows are built by the walk of the fused path, so the CSR solve must
equal the fused solve up to the order of FP32 atomics, and both match the
FP64 oracle; the packed form carries 16-bit chords (fixed point of the voxel
diagonal, or FP16), and its RSP error against the oracle is measured and
bounded for each code.
"""
import numpy as np
import pytest
import torch

import oracle as O
import paper_1802_01070_b300 as pct
from tests import parity_util as U

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def tiny(cuda_device):
    cfg, rsp, hull, hist = U.scan("tiny")
    geo, rowptr, j, ln, margin, A, cond = U.oracle_rows("tiny")
    ctx = U.context(cfg, hull, hist)
    yield dict(cfg=cfg, hull=hull, hist=hist, A=A, rowptr=rowptr, j=j, ctx=ctx)
    ctx.close()


def _solve(ctx, hull, mode, iters, lam, block):
    ctx.set_option(pct.PCT_OPT_MODE, mode)
    x = torch.from_numpy(hull.astype(np.float32)).cuda()
    ctx.solve(x, iters, lam, block)
    ctx.synchronize()
    return x.cpu().numpy().astype(np.float64)


def test_csr_rows_are_the_fused_rows(tiny):
    ctx = tiny["ctx"]
    ctx.set_option(pct.PCT_OPT_MODE, pct.PCT_MODE_CSR)
    ctx.build_rows()
    ctx.synchronize()
    _, _, nnz = ctx.rows(0, ctx.n, max_nnz=256)
    assert int(ctx.stat(pct.PCT_STAT_ROW_ENTRIES)) == int(nnz.sum().item())
    assert ctx.stat(pct.PCT_STAT_ROW_BYTES) >= 8 * ctx.stat(pct.PCT_STAT_ROW_ENTRIES)


@pytest.mark.parametrize("lam", [1e-4, 0.5])
def test_csr_solve_equals_fused_solve_and_oracle(tiny, lam):
    cfg, ctx, hull = tiny["cfg"], tiny["ctx"], tiny["hull"]
    xf = _solve(ctx, hull, pct.PCT_MODE_FUSED, cfg.iters, lam, cfg.block)
    xc = _solve(ctx, hull, pct.PCT_MODE_CSR, cfg.iters, lam, cfg.block)
    hm = hull.astype(bool)
    assert np.max(np.abs(xc - xf)[hm] / np.abs(xf)[hm]) <= 1e-4
    xo = O.drop(tiny["A"], tiny["hist"]["wepl"].astype(np.float64), cfg.iters, lam, cfg.block,
                hull.astype(np.float64))
    rel = np.abs(xc - xo)[hm] / np.abs(xo)[hm]
    assert (rel <= 1e-3).mean() >= 0.99 and rel.mean() <= 1e-4


@pytest.mark.parametrize("code", ["fixed16", "fp16"])
def test_packed_solve_error_against_fp64(tiny, code):
    cfg, ctx, hull = tiny["cfg"], tiny["ctx"], tiny["hull"]
    ctx.set_option(pct.PCT_OPT_CHORD_CODE,
                   pct.PCT_CHORD_FIXED16 if code == "fixed16" else pct.PCT_CHORD_FP16)
    xp = _solve(ctx, hull, pct.PCT_MODE_PACKED, cfg.iters, 0.5, cfg.block)
    entries = int(ctx.stat(pct.PCT_STAT_ROW_ENTRIES))
    nbytes = ctx.stat(pct.PCT_STAT_ROW_BYTES)
    xf = _solve(ctx, hull, pct.PCT_MODE_FUSED, cfg.iters, 0.5, cfg.block)
    ctx.set_option(pct.PCT_OPT_CHORD_CODE, pct.PCT_CHORD_FIXED16)
    xo = O.drop(tiny["A"], tiny["hist"]["wepl"].astype(np.float64), cfg.iters, 0.5, cfg.block,
                hull.astype(np.float64))
    hm = hull.astype(bool)
    rp = np.abs(xp - xo)[hm] / np.abs(xo)[hm]
    rf = np.abs(xf - xo)[hm] / np.abs(xo)[hm]
    print("packed (%s chords): %d entries, %.2f B/entry; rel err vs FP64 max %.3g mean %.3g "
          "(fused: max %.3g mean %.3g)" % (code, entries, nbytes / max(entries, 1), rp.max(), rp.mean(),
                                           rf.max(), rf.mean()))
    if code == "fp16":
        # FP16 chords carry a relative rounding of up to 2^-11: the RSP moves by about that much
        assert rp.mean() <= 5e-4 and (rp <= 1e-2).mean() >= 0.999
    else:
        # fixed-point chords (~1.7e-5 mm) keep the FP32 path's accuracy
        assert rp.mean() <= 2e-5 and (rp <= 1e-3).mean() >= 0.999 and rp.max() <= 1e-2
    assert nbytes / max(entries, 1) < 4.0
    # packed rows keep runs outside the hull too: at least as many entries as CSR rows
    assert entries >= tiny["rowptr"][-1] - 1000


def test_chord_code_option(cuda_device):
    cfg, rsp, hull, hist = U.scan("tiny")
    h = {k: np.ascontiguousarray(v[:3000]) for k, v in hist.items()}
    ctx = U.context(cfg, hull, h)
    assert ctx.get_option(pct.PCT_OPT_CHORD_CODE) == pct.PCT_CHORD_FIXED16
    with pytest.raises(pct.PctError) as e:
        ctx.set_option(pct.PCT_OPT_CHORD_CODE, 7)
    assert e.value.status == pct.PCT_ERR_ARG
    ctx.set_option(pct.PCT_OPT_MODE, pct.PCT_MODE_PACKED)
    ctx.build_rows()
    assert ctx.stat(pct.PCT_STAT_ROW_ENTRIES) > 0
    ctx.set_option(pct.PCT_OPT_CHORD_CODE, pct.PCT_CHORD_FP16)
    assert ctx.stat(pct.PCT_STAT_ROW_ENTRIES) == 0          # a new chord code drops packed rows
    assert ctx.get_option(pct.PCT_OPT_CHORD_CODE) == pct.PCT_CHORD_FP16
    ctx.close()


def test_stored_rows_ragged_blocks_and_invalidation(cuda_device):
    cfg, rsp, hull, hist = U.scan("tiny")
    h = {k: np.ascontiguousarray(v[:10007]) for k, v in hist.items()}
    geo = U.geometry(cfg, hull)
    rowptr, j, ln, margin = O.rows(geo, h)
    A = O.csr(rowptr, j, ln, geo.n_vox)
    xo = O.drop(A, h["wepl"].astype(np.float64), 2, 0.5, 1000, hull.astype(np.float64))
    ctx = U.context(cfg, hull, h)
    hm = hull.astype(bool)
    for mode in (pct.PCT_MODE_CSR, pct.PCT_MODE_PACKED):
        x = _solve(ctx, hull, mode, 2, 0.5, 1000)
        rel = np.abs(x - xo)[hm] / xo[hm]
        assert (rel <= (1e-3 if mode == pct.PCT_MODE_CSR else 1e-2)).mean() >= 0.999, mode
        assert ctx.stat(pct.PCT_STAT_ROW_ENTRIES) > 0
    ctx.set_option(pct.PCT_OPT_MODE, pct.PCT_MODE_FUSED)
    assert ctx.stat(pct.PCT_STAT_ROW_ENTRIES) == 0          # mode change drops stored rows
    ctx.set_option(pct.PCT_OPT_MODE, pct.PCT_MODE_CSR)
    ctx.build_rows()
    assert ctx.stat(pct.PCT_STAT_ROW_ENTRIES) > 0
    ctx.load_histories({k: torch.from_numpy(v).cuda() for k, v in h.items()})
    assert ctx.stat(pct.PCT_STAT_ROW_ENTRIES) == 0          # reload drops stored rows
    x = _solve(ctx, hull, pct.PCT_MODE_CSR, 2, 0.5, 1000)  # rebuilt on demand
    assert (np.abs(x - xo)[hm] / xo[hm] <= 1e-3).mean() >= 0.999
    ctx.close()
