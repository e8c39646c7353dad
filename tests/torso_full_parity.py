"""Full-size torso reconstruction against the FP64 oracle (a long run, not a pytest test).

The torso scan (280x280x96 grid of 1 mm voxels, 1.16e8 protons, 180 angles)
solved by DROP with blocks of 320000 protons (Sec. IV-B, the paper's setting
for its simulated data), from x0 = 1 inside the hull, on the GPU and by the
oracle block by block on the host cores (rows of one block at a time, x kept
between blocks, as the Gauss-Seidel sequence of blocks requires).  Reported:

* free-running: every hull voxel of the two final volumes (each side on its own
  trajectory) -- the share within 1e-3 relative, mean, quantiles, maximum;
* teacher-forced: for sampled blocks, the GPU's block step from its own x
  against the oracle's step from the same x, on the voxels the comparison
  rule of oracle/compare.py keeps (the step's arithmetic alone);
* row-forced: a third trajectory, the oracle's FP64 DROP arithmetic on the
  GPU's own rows (voxel indices and FP32 chords read back block by block).
  GPU against it isolates the FP32 solve arithmetic; it against the oracle
  isolates the rows (FP32 paths resolving near-face crossings differently).

Usage (GPU machine; one full iteration takes the oracle ~30-40 min on 16 cores):
    python tests/torso_full_parity.py --iters 1 --every 24 --out torso_parity.json
Writes the JSON summary after every sampled block, so a cut-short run keeps
what it measured.
"""
from __future__ import annotations

import argparse
import json
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402
import torch  # noqa: E402

import oracle as O  # noqa: E402
import paper_1802_01070_b300 as pct  # noqa: E402
import synth  # noqa: E402
from oracle.compare import Exclusion, solve_parity  # noqa: E402


def _stats(xg, xo, hm):
    rel = np.abs(xg - xo)[hm] / np.maximum(np.abs(xo[hm]), 1e-30)
    q = np.quantile(rel, [0.5, 0.99, 0.999, 0.9999])
    return {"hull_voxels": int(hm.sum()), "frac_within_1e-3": float((rel <= 1e-3).mean()),
            "frac_within_1e-4": float((rel <= 1e-4).mean()), "mean_rel": float(rel.mean()),
            "median_rel": float(q[0]), "p99_rel": float(q[1]), "p999_rel": float(q[2]),
            "p9999_rel": float(q[3]), "max_rel": float(rel.max())}


def _exclusion(ctx, rowptr, j, ln, margin, cond, n_vox, block, x, b):
    ex = Exclusion(n_vox, block, x=x, b=b)
    n = ctx.n
    for a in range(0, n, 8192):
        k = min(n, a + 8192) - a
        _, _, nnz = ctx.rows(a, k, max_nnz=0)
        W = max(int(nnz.max().item()), 1)
        gi, gl, gn = ctx.rows(a, k, max_nnz=W)
        e0, e1 = int(rowptr[a]), int(rowptr[a + k])
        ex.add(a, gi.cpu().numpy(), gl.cpu().numpy(), gn.cpu().numpy(), rowptr[a:a + k + 1] - e0,
               j[e0:e1], ln[e0:e1], margin[a:a + k], cond[a:a + k])
    return ex.finish()


def _gpu_csr(ctx, n_vox, chunk=8192):
    """The GPU's rows of the protons loaded in ctx as an FP64 CSR matrix."""
    n = ctx.n
    counts, js, ls = [], [], []
    for a in range(0, n, chunk):
        k = min(n, a + chunk) - a
        _, _, nnz = ctx.rows(a, k, max_nnz=0)
        W = max(int(nnz.max().item()), 1)
        gi, gl, gn = ctx.rows(a, k, max_nnz=W)
        gi, gl, gn = gi.cpu().numpy(), gl.cpu().numpy(), gn.cpu().numpy().astype(np.int64)
        keep = np.arange(W)[None, :] < gn[:, None]
        counts.append(gn)
        js.append(gi[keep])
        ls.append(gl[keep].astype(np.float64))
    rowptr = np.concatenate([[0], np.cumsum(np.concatenate(counts))])
    return O.csr(rowptr, np.concatenate(js), np.concatenate(ls), n_vox)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--iters", type=int, default=1)
    ap.add_argument("--every", type=int, default=24, help="teacher-force every n-th block")
    ap.add_argument("--blocks", type=int, default=0, help="stop after this many blocks (0: all)")
    ap.add_argument("--out", default="torso_parity.json")
    ap.add_argument("--no-row-forced", action="store_true", help="skip the FP64 solve on the GPU's rows")
    args = ap.parse_args()
    t_start = time.time()
    cfg = synth.CONFIGS["torso"]
    B, lam = cfg.block, cfg.lam
    rsp, hull = synth.phantom(cfg)
    hull_np = hull.numpy()
    hm = hull_np.astype(bool)
    hist = synth.histories(cfg, "cuda", chunk=1 << 24, rsp=rsp)
    n = cfg.n_protons
    nb = (n + B - 1) // B
    if args.blocks:
        nb = min(nb, args.blocks)
    geo = O.Geometry(cfg.shape, (cfg.voxel,) * 3, cfg.origin, mask=hull_np)
    x0 = hull_np.astype(np.float64)
    xg = torch.from_numpy(hull_np.astype(np.float32)).cuda()
    xo = x0.copy()
    xr = None if args.no_row_forced else x0.copy()
    out = {"workload": "torso 280x280x96, 1.16e8 protons, block %d, lambda %g, %d iteration(s), %d blocks "
                       "per iteration" % (B, lam, args.iters, nb),
           "oracle_threads": O.num_threads(), "teacher_forced": []}
    with pct.Context(cfg.shape, cfg.voxel, cfg.origin, hull=hull_np) as ck:
        for it in range(args.iters):
            for k in range(nb):
                a = k * B
                m = min(n, a + B) - a
                sub = {kk: v[a:a + m] for kk, v in hist.items()}
                ck.load_histories(sub)
                forced = (k % args.every == 0)
                x_before = xg.cpu().numpy().astype(np.float64) if forced else None
                ck.solve(xg, 1, lam, B)
                ck.synchronize()
                sub_np = {kk: v.cpu().numpy() for kk, v in sub.items()}
                if forced:
                    rowptr, j, ln, margin, cond = O.rows(geo, sub_np, with_cond=True)
                else:
                    rowptr, j, ln, margin = O.rows(geo, sub_np)
                A = O.csr(rowptr, j, ln, geo.n_vox)
                b = sub_np["wepl"].astype(np.float64)
                xo = O.drop(A, b, 1, lam, B, xo)
                if xr is not None:
                    Ag = _gpu_csr(ck, geo.n_vox)
                    xr = O.drop(Ag, b, 1, lam, B, xr)
                    del Ag
                if forced:
                    xt = O.drop(A, b, 1, lam, B, x_before)
                    ex = _exclusion(ck, rowptr, j, ln, margin, cond, geo.n_vox, B, x_before, b)
                    r = solve_parity(xg.cpu().numpy(), xt, hull_np, ex)
                    r.update(iteration=it + 1, block=k)
                    out["teacher_forced"].append(r)
                    out["teacher_forced_clean_max"] = max(q["clean_max"] for q in out["teacher_forced"])
                    out["teacher_forced_unexcused_rows"] = sum(q["rows_unexcused"] for q in out["teacher_forced"])
                    out["blocks_done"] = it * nb + k + 1
                    out["free_running_so_far"] = _stats(xg.cpu().numpy().astype(np.float64), xo, hm)
                    if xr is not None:
                        out["row_forced_so_far"] = {
                            "gpu_vs_fp64_on_gpu_rows": _stats(xg.cpu().numpy().astype(np.float64), xr, hm),
                            "fp64_on_gpu_rows_vs_oracle": _stats(xr, xo, hm)}
                    out["elapsed_s"] = time.time() - t_start
                    with open(args.out, "w") as f:
                        json.dump(out, f, indent=1)
                    print("iteration %d block %d/%d: teacher-forced clean max %.3g; free-running within 1e-3 "
                          "%.6f (%.0f s)" % (it + 1, k + 1, nb, r["clean_max"],
                                             out["free_running_so_far"]["frac_within_1e-3"], out["elapsed_s"]),
                          flush=True)
                del A, rowptr, j, ln
    out["blocks_done"] = args.iters * nb
    out["free_running"] = _stats(xg.cpu().numpy().astype(np.float64), xo, hm)
    if xr is not None:
        out["row_forced"] = {"gpu_vs_fp64_on_gpu_rows": _stats(xg.cpu().numpy().astype(np.float64), xr, hm),
                             "fp64_on_gpu_rows_vs_oracle": _stats(xr, xo, hm)}
    truth = rsp.numpy().astype(np.float64)
    out["rsp_err_vs_truth"] = {"gpu_mean_abs_rel": float((np.abs(xg.cpu().numpy() - truth)[hm] / truth[hm]).mean()),
                               "oracle_mean_abs_rel": float((np.abs(xo - truth)[hm] / truth[hm]).mean())}
    out["elapsed_s"] = time.time() - t_start
    with open(args.out, "w") as f:
        json.dump(out, f, indent=1)
    print(json.dumps({k: v for k, v in out.items() if k != "teacher_forced"}))
    # asserted: every sampled block step (teacher-forced) and the FP32 solve
    # arithmetic over the whole run (row-forced); the free-running share is
    # reported: near-face rows resolved differently feed every later block
    ok = out["teacher_forced_clean_max"] <= 1e-3 and out["teacher_forced_unexcused_rows"] == 0
    if xr is not None:
        ok = ok and out["row_forced"]["gpu_vs_fp64_on_gpu_rows"]["frac_within_1e-3"] >= 0.999
    return 0 if ok else 1


if __name__ == "__main__":
    sys.exit(main())
