#!/usr/bin/env python
"""Throughput of the fused MLP -> voxel walk -> DROP reconstruction on B300.

Workload (default): torso-sized scan, 280x280x96 grid of 1 mm voxels, 1.16e8
synthetic protons over 180 gantry angles in 2-degree steps, 6 DROP iterations,
block size 320000, rows recomputed on the fly (A never stored), FP32.
One step = one reconstruction from the device-resident histories: load them
(device-to-device copy), then pct_solve from the initial iterate (x0 = 1 inside
the hull): per-proton records (hull entry/exit) and valid-proton lists, then 6
iterations of per-block fused MLP + walk + dot + scatter and the block apply.
With --mode csr|packed a step is the solve over rows built once beforehand
(the build is timed apart: row_build_s).

Prints ONE JSON line (rank 0).  `value` is proton-rows/s per iteration (rows =
protons whose path crosses the hull), summed over ranks; `recon_s` is the
seconds of one reconstruction; `e2e` repeats the metric through the C ABI with
host buffers (history upload and result download inside the timed region).
`--impl reference` times the FP64 CPU oracle instead (bounded sample).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "proton-rows/s per iteration and recon seconds at 116M protons; RSP err vs FP64"
UNIT = "proton-rows/s"


def _args():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=3)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--config", default="torso")
    p.add_argument("--protons", type=int, default=None, help="override the proton count")
    p.add_argument("--block", type=int, default=None)
    p.add_argument("--cta", type=int, default=None)
    p.add_argument("--task", default="drop",
                   choices=["drop", "adam", "batch", "blocks", "fbp", "clean", "regions"],
                   help="drop: DROP reconstruction (default); adam: TV-regularised Adam "
                        "reconstruction with the differentiable projector (workload 'diff')")
    p.add_argument("--mode", default="fused", choices=["fused", "csr", "packed"],
                   help="row form: recomputed on the fly, or stored (built once, timed apart)")
    p.add_argument("--walk", default=None, choices=["rounds", "lanes"],
                   help="walk of the fused DROP step (default: the library's, lanes)")
    p.add_argument("--persistent-block", type=int, default=None,
                   help="largest block size solved in one persistent launch (0: never; default: the "
                        "library's, 0)")
    p.add_argument("--chord", default="fixed16", choices=["fixed16", "fp16"],
                   help="chord code of the packed rows")
    p.add_argument("--cpu-sample", type=int, default=320000)
    p.add_argument("--ref-sample", type=int, default=100000)
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-e2e", action="store_true")
    return p.parse_args()


# ----------------------------------------------------------------------------
# clocks during the timed region
# ----------------------------------------------------------------------------

class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
    NAMES = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")

    def __init__(self, pci=None):
        self.pci = pci
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        cmd = ["nvidia-smi", "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits",
               "-lms", "200"]
        if self.pci:
            cmd += ["-i", self.pci]
        try:
            self.proc = subprocess.Popen(cmd, stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, power, reasons = [], [], [], set()
        for line in open(self.path):
            f = [v.strip() for v in line.split(",")]
            if len(f) < 8:
                continue
            try:
                sm.append(float(f[0]))
                smax.append(float(f[1]))
                power.append(float(f[2]))
            except ValueError:
                continue
            for name, v in zip(self.NAMES, f[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(name)
        os.unlink(self.path)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        load = [s for s, p in zip(sm, power) if p > 200.0] or sm
        return {"sm_mhz": statistics.median(load), "sm_max_mhz": max(smax),
                "power_w_max": max(power), "samples": len(sm), "reasons": sorted(reasons)}


def _pci_id(torch, dev):
    try:
        p = torch.cuda.get_device_properties(dev)
        return "%08x:%02x:%02x.0" % (p.pci_domain_id, p.pci_bus_id, p.pci_device_id)
    except Exception:
        return None


# ----------------------------------------------------------------------------
# algorithmic work model of the fused kernel (FP32 flops, FMA = 2)
# ----------------------------------------------------------------------------
FLOP_PER_SAMPLE = 103   # one MLP sample: Sigma2 moments, Highland factor, 2x2 Kalman gain, 2 planes
FLOP_PER_SEGMENT = 25   # segment set-up of the voxel walk (direction, length, first crossings)
FLOP_PER_VISIT = 16     # one face crossing, the dot and norm FMAs, the scatter product


def fused_flops(n_valid, mean_pts, mean_nnz):
    """Algorithmic FP32 flops of one DROP pass over n_valid rows: each row's MLP
    samples, walk segments and visits once (the scatter reuses the walk)."""
    samples = max(mean_pts - 2.0, 0.0)
    segs = max(mean_pts - 1.0, 0.0)
    return (samples * FLOP_PER_SAMPLE + segs * FLOP_PER_SEGMENT + mean_nnz * FLOP_PER_VISIT) * n_valid


# the sources the fused block kernel is compiled from (host code excluded)
KERNEL_SOURCES = ("pct_device.cuh", "pct_kernels.cu", "pct_warp.cuh", "pct_round.cuh")


def _kernel_hash():
    h = hashlib.sha256()
    d = os.path.join(ROOT, "paper_1802_01070_b300", "csrc")
    for f in KERNEL_SOURCES:
        h.update(open(os.path.join(d, f), "rb").read())
    return h.hexdigest()[:16]


def _profiled_traffic(workload):
    """The committed ncu summary of the fused kernel (DRAM bytes per valid row,
    issue rate), if it was taken on the current kernel source; else None."""
    path = os.path.join(ROOT, "profiles", "drop_fused_traffic.json")
    try:
        d = json.load(open(path))
    except (OSError, ValueError):
        return None
    if d.get("kernel_hash") != _kernel_hash():
        return None
    per_row = d.get("dram_bytes_per_valid_row")
    return d if per_row else None


def measured_ceilings(pct, device, n_slots):
    """(FP32 TFLOP/s, 1e9 float2 atomics/s) measured now by the library's
    microbenchmarks on ``device``; the atomic array has the DROP accumulator's
    size."""
    tf, _ = pct.pct_peak_fp32(device, repeats=5)
    ga, _ = pct.pct_peak_atomic(n_slots, device, repeats=5)
    return tf, ga


def _measured_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        return {}


# ----------------------------------------------------------------------------
# Multi-rank aggregation: every rank runs an independent replica of the scan
# (the solve does not shard), the job's time is its slowest rank's
# ----------------------------------------------------------------------------

def max_over_ranks(value, dist=None):
    """Largest `value` over all ranks of the process group (itself at N = 1)."""
    if dist is None:
        return value
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_throughput(world, units_per_rank, seconds):
    """Whole-job throughput of `world` replicas that each process `units_per_rank`."""
    return world * units_per_rank / seconds


# ----------------------------------------------------------------------------
# CPU oracle leg (test infrastructure; timed as it stands)
# ----------------------------------------------------------------------------

def oracle_solve_timed(cfg, hull_np, hist_np, iters, lam, block):
    import numpy as np

    import oracle as O
    geo = O.Geometry(cfg.shape, (cfg.voxel,) * 3, cfg.origin, mask=hull_np)
    t0 = time.perf_counter()
    rowptr, j, ln, _ = O.rows(geo, hist_np)
    A = O.csr(rowptr, j, ln, geo.n_vox)
    x = O.drop(A, hist_np["wepl"].astype(np.float64), iters, lam, block, hull_np.astype(np.float64))
    dt = time.perf_counter() - t0
    valid = int(np.count_nonzero(np.diff(rowptr)))
    return x, dt, valid, O.num_threads()


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    import numpy as np

    import synth
    cfg = synth.CONFIGS[args.config]
    n = min(args.ref_sample, cfg.n_protons)
    rsp, hull = synth.phantom(cfg)
    hist = synth.to_numpy(synth.histories(cfg, "cpu", n=n, rsp=rsp))
    hull_np = hull.numpy()
    block = args.block or cfg.block
    times, valid, threads = [], 0, 1
    for k in range(args.warmup + args.steps):
        _, dt, valid, threads = oracle_solve_timed(cfg, hull_np, hist, cfg.iters, cfg.lam, block)
        if k >= args.warmup:
            times.append(dt)
    t = statistics.mean(times)
    value = valid * cfg.iters / t
    sample = ("first %d protons of the %s scan (%d cross the hull), full %d-iteration DROP "
              "solve with rows built once, block %d" % (n, cfg.name, valid, cfg.iters, block))
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": t * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": _config(cfg, block, cfg.n_protons),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))
    return 0


FORM_TEXT = {"fused": "fused on-the-fly MLP+walk (A never stored)",
             "csr": "rows stored as CSR (int32 voxel + FP32 chord per entry), built once",
             "packed": "rows stored packed (1-byte step code + 16-bit chord per entry), built once"}


def _config(cfg, block, n, mode="fused"):
    return {"workload": "%s: %dx%dx%d grid of %g mm voxels, %d protons over %d angles, %d DROP "
                        "iterations, block %d, %s"
                        % (cfg.name, *cfg.shape, cfg.voxel, n, cfg.n_angles, cfg.iters, block,
                           FORM_TEXT[mode]),
            "grid": list(cfg.shape), "voxel_mm": cfg.voxel, "protons": n, "angles": cfg.n_angles,
            "iters": cfg.iters, "block": block, "lambda": cfg.lam, "x0": "1.0 inside hull",
            "l2": "inputs larger than L2: 48 B of history per proton read each step and 72 B of "
                  "record + list entry per crossing proton streamed each iteration (%.1f GB of "
                  "histories and records)" % (n * 112 / 1e9)}


# ----------------------------------------------------------------------------
# GPU leg
# ----------------------------------------------------------------------------

def run_ours(args):
    import numpy as np
    import torch

    import paper_1802_01070_b300 as pct
    import synth

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("gloo")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    cfg = synth.CONFIGS[args.config]
    n = args.protons or cfg.n_protons
    if n != cfg.n_protons:
        cfg = synth.scaled(cfg, n)
    block = args.block or cfg.block
    rsp, hull = synth.phantom(cfg)
    hull_np = hull.numpy()
    hist = synth.histories(cfg, dev, chunk=1 << 24, rsp=rsp)
    s_cpu = min(args.cpu_sample, n)
    sample_hist = {k: v[:s_cpu].clone() for k, v in hist.items()}
    torch.cuda.synchronize(dev)

    ctx = pct.Context(cfg.shape, cfg.voxel, cfg.origin, hull=hull_np, device=local)
    if args.cta:
        ctx.set_option(pct.PCT_OPT_CTA_THREADS, args.cta)
    mode = {"fused": pct.PCT_MODE_FUSED, "csr": pct.PCT_MODE_CSR, "packed": pct.PCT_MODE_PACKED}[args.mode]
    ctx.set_option(pct.PCT_OPT_MODE, mode)
    ctx.set_option(pct.PCT_OPT_CHORD_CODE,
                   pct.PCT_CHORD_FIXED16 if args.chord == "fixed16" else pct.PCT_CHORD_FP16)
    if args.walk:
        ctx.set_option(pct.PCT_OPT_WALK, {"rounds": pct.PCT_WALK_ROUNDS, "lanes": pct.PCT_WALK_LANES}[args.walk])
    walk = ctx.get_option(pct.PCT_OPT_WALK)
    if args.persistent_block is not None:
        ctx.set_option(pct.PCT_OPT_PERSISTENT_BLOCK, args.persistent_block)
    ctx.load_histories(hist)
    build_s = None
    if mode != pct.PCT_MODE_FUSED:
        torch.cuda.synchronize(dev)
        tb = time.perf_counter()
        ctx.build_rows()
        ctx.synchronize()
        build_s = time.perf_counter() - tb

    # rows crossing the hull, and the mean path size of a sample (work model)
    valid = 0
    for a in range(0, n, 1 << 22):
        c = min(n, a + (1 << 22)) - a
        valid += int((ctx.hull_states(a, c)[:, 10] > 0.5).sum().item())
    ns = min(n, 65536)
    _, npts = ctx.mlp(0, ns, max_pts=1024)
    _, _, nnz = ctx.rows(0, ns, max_nnz=2048)
    ok = npts > 0
    mean_pts = float(npts[ok].float().mean().item()) if ok.any() else 0.0
    mean_nnz = float(nnz[ok].float().mean().item()) if ok.any() else 0.0

    x0 = torch.from_numpy(hull_np.astype(np.float32)).to(dev)
    x = torch.empty_like(x0)

    # fused: one step = one reconstruction from the device-resident histories:
    # load them (device-to-device copy; the library then recomputes the
    # per-proton records it keeps between calls) and solve from x0.  Stored
    # rows: one step = the solve over the rows built once (build timed apart).
    def step():
        if mode == pct.PCT_MODE_FUSED:
            ctx.load_histories(hist)
        x.copy_(x0)
        ctx.solve(x, cfg.iters, cfg.lam, block)

    for _ in range(args.warmup):
        step()
    ctx.synchronize()

    pci = _pci_id(torch, dev)
    clk = ClockSampler(pci)
    ctx.reset_stats()
    # time every k-th launch of the block kernel inside the timed region: about
    # 256 launches per solve, so the event records do not slow a solve of many
    # small blocks
    blocks_per_solve = cfg.iters * math.ceil(n / block)
    ctx.set_option(pct.PCT_OPT_TIMING, max(1, blocks_per_solve // 256))
    stream = torch.cuda.current_stream(dev)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    if dist:
        dist.barrier()
    torch.cuda.synchronize(dev)
    clk.start()
    time.sleep(0.3)
    e0.record(stream)
    for _ in range(args.steps):
        step()
    e1.record(stream)
    torch.cuda.synchronize(dev)
    clocks = clk.stop()
    ctx.synchronize()
    if dist:
        dist.barrier()
    step_ms = e0.elapsed_time(e1) / args.steps
    launches = int(ctx.stat(pct.PCT_STAT_LAUNCHES))
    fused_ms = ctx.stat(pct.PCT_STAT_FUSED_MS)
    fused_n = int(ctx.stat(pct.PCT_STAT_FUSED_LAUNCHES))
    timed_n = int(ctx.stat(pct.PCT_STAT_TIMED_LAUNCHES))
    ctx.set_option(pct.PCT_OPT_TIMING, 0)
    ctx.reset_stats()
    step_ms = max_over_ranks(step_ms, dist)
    value = replica_throughput(world, valid * cfg.iters, step_ms * 1e-3)

    # roofline of the dominant kernel (fused DROP block step)
    peaks = _measured_peaks()
    fp32_peak, atomic_peak = measured_ceilings(pct, local, cfg.n_vox)
    avg_launch_s = fused_ms * 1e-3 / max(timed_n, 1)
    persistent = timed_n == 0 and args.mode == "fused"
    if persistent:
        # one persistent launch per solve: the average block step (walk,
        # barriers and apply) from the step time
        avg_launch_s = step_ms * 1e-3 / blocks_per_solve
    blocks_per_iter = math.ceil(n / block)
    flops_launch = fused_flops(valid, mean_pts, mean_nnz) / blocks_per_iter
    achieved = flops_launch / avg_launch_s / 1e12
    hbm_bytes_launch = (n / blocks_per_iter) * (16 * 4)        # proton records streamed per launch
    prof = _profiled_traffic(cfg.name) if args.mode == "fused" else None
    per_row_traffic = prof["dram_bytes_per_valid_row"] if prof else None
    roofline = {"bound": "alu", "achieved": achieved, "peak": fp32_peak, "unit": "TFLOP/s",
                "frac": achieved / fp32_peak,
                "traffic": (per_row_traffic * valid / blocks_per_iter) if per_row_traffic else None,
                "kernel": ("k_drop_batch (one persistent launch per solve; per block step incl. "
                           "barriers and apply)") if persistent else
                          ("k_drop_rounds" if walk == pct.PCT_WALK_ROUNDS else "k_drop_fused"),
                "avg_launch_ms": avg_launch_s * 1e3,
                "launches_timed": timed_n, "launches": fused_n,
                "peak_source": "measured: pct_peak_fp32, FP32 FMA loop filling every SM (best of 5, "
                               "CUDA events), in this run",
                "atomic": {"achieved_g_per_s": valid * mean_nnz / blocks_per_iter / avg_launch_s / 1e9,
                           "peak_g_per_s": atomic_peak,
                           "frac": valid * mean_nnz / blocks_per_iter / avg_launch_s / 1e9 / atomic_peak,
                           "peak_source": "measured: pct_peak_atomic, float2 atomicAdd to uniformly "
                                          "hashed slots of a %d-slot array (the accumulator's size, "
                                          "L2-resident), in this run" % cfg.n_vox,
                           "model": "one float2 atomic per visit (%.1f visits per valid row)" % mean_nnz},
                "flops_model": "(%.1f MLP samples x %d + %.1f segments x %d + %.1f visits x %d) "
                               "per valid row" % (max(mean_pts - 2, 0), FLOP_PER_SAMPLE,
                                                  max(mean_pts - 1, 0), FLOP_PER_SEGMENT, mean_nnz,
                                                  FLOP_PER_VISIT),
                "issue_frac_profiled": (prof["issue_ipc_per_sm"] / prof["issue_ipc_peak"]
                                        if prof and "issue_ipc_per_sm" in prof else None),
                "issue_note": "the kernel is bound by instruction issue (integer/compare/branch work "
                              "of the voxel walk), not FP32 math: issued warp instructions per SM "
                              "cycle over the 4 the SM can issue, from the committed ncu capture of "
                              "this kernel source",
                "hbm_gbs_algorithmic": hbm_bytes_launch / avg_launch_s / 1e9,
                "hbm_peak_gbs": peaks.get("hbm_gbs"),
                "hbm_frac_algorithmic": (hbm_bytes_launch / avg_launch_s / 1e9 / peaks["hbm_gbs"]
                                         if peaks.get("hbm_gbs") else None),
                "fused_share_of_step": avg_launch_s * 1e3 * fused_n / args.steps / step_ms
                if step_ms else None}
    if args.mode != "fused":
        # stored rows stream from HBM: entry bytes (8 CSR, 3 packed) + row offset + WEPL per row
        entries = ctx.stat(pct.PCT_STAT_ROW_ENTRIES)
        per_entry = 8.0 if args.mode == "csr" else 3.0
        per_row = 8.0 + 4.0 + (8.0 if args.mode == "packed" else 0.0)
        bytes_launch = (entries * per_entry + n * per_row) / blocks_per_iter
        hbm_peak = float(peaks.get("hbm_gbs", 6400.0))
        ach = bytes_launch / avg_launch_s / 1e9
        roofline = {"bound": "hbm", "achieved": ach, "peak": hbm_peak, "unit": "GB/s",
                    "frac": ach / hbm_peak, "traffic": None,
                    "kernel": "k_drop_csr" if args.mode == "csr" else "k_drop_packed",
                    "avg_launch_ms": avg_launch_s * 1e3, "launches_timed": timed_n, "launches": fused_n,
                    "bytes_model": "%.0f B/entry x %.4g entries + %.0f B/row, per iteration" % (
                        per_entry, entries, per_row),
                    "peak_source": "MEASURED_PEAKS hbm_gbs (copy bandwidth)",
                    "fused_share_of_step": avg_launch_s * 1e3 * fused_n / args.steps / step_ms
                    if step_ms else None}

    out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": step_ms, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
           "config": dict(_config(cfg, block, n, args.mode), mode=args.mode,
                          **({"chord": args.chord} if args.mode == "packed" else {})),
           "recon_s": step_ms * 1e-3,
           "row_build_s": build_s, "row_bytes": ctx.stat(pct.PCT_STAT_ROW_BYTES),
           "row_entries": ctx.stat(pct.PCT_STAT_ROW_ENTRIES),
           "rows_in_hull": valid, "mean_nnz_per_row": mean_nnz, "mean_mlp_points": mean_pts,
           "roofline": roofline, "gpu_launches": launches, "clocks": clocks}

    # end to end through the C ABI with pinned host buffers
    if not args.no_e2e:
        host = {k: v.cpu().pin_memory() for k, v in hist.items()}
        xh = torch.from_numpy(hull_np.astype(np.float32)).pin_memory()
        del hist
        torch.cuda.empty_cache()
        h2d = sum(v.numel() * 4 for v in host.values()) + xh.numel() * 4
        times = []
        for k in range(3):
            xw = xh.clone().pin_memory()
            torch.cuda.synchronize(dev)
            t0 = time.perf_counter()
            ctx.load_histories(host)
            ctx.solve_host(xw.numpy(), cfg.iters, cfg.lam, block)
            times.append(time.perf_counter() - t0)
        te = max_over_ranks(statistics.mean(times[1:]), dist)
        out["e2e"] = {"value": replica_throughput(world, valid * cfg.iters, te), "unit": UNIT,
                      "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": xh.numel() * 4,
                      "recon_s": te}
    else:
        del hist

    # CPU oracle baseline and FP64 parity on a bounded sample (rank 0, N = 1)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        s = s_cpu
        sub = sample_hist
        sub_np = synth.to_numpy(sub)
        xo, dt, vs, threads = oracle_solve_timed(cfg, hull_np, sub_np, cfg.iters, cfg.lam, block)
        with pct.Context(cfg.shape, cfg.voxel, cfg.origin, hull=hull_np, device=local) as c2:
            c2.set_option(pct.PCT_OPT_MODE, mode)
            c2.set_option(pct.PCT_OPT_CHORD_CODE, ctx.get_option(pct.PCT_OPT_CHORD_CODE))
            c2.load_histories(sub)
            xg = torch.from_numpy(hull_np.astype(np.float32)).to(dev)
            c2.solve(xg, cfg.iters, cfg.lam, block)
            c2.synchronize()
            xg = xg.cpu().numpy().astype(np.float64)
        ex = exclusion_voxels(pct, cfg, hull_np, sub, sub_np, local, block)
        from oracle.compare import solve_parity
        par = solve_parity(xg, xo, hull_np, ex)
        out["cpu_baseline"] = {"value": vs * cfg.iters / dt, "unit": UNIT, "cores": threads,
                               "kind": "oracle",
                               "sample": "first %d protons (%d cross the hull): rows built once, "
                                         "%d DROP iterations, block %d, FP64, %.1f s"
                                         % (s, vs, cfg.iters, block, dt)}
        out["rsp_err_vs_fp64"] = dict(
            par, sample="same %d-proton sample, GPU FP32 %s vs oracle FP64; 'clean' = hull voxels the "
                        "comparison rule keeps: DROP count s_j identical on both sides in every block, "
                        "and no row crossing the voxel with chords that differ by more than 2e-3 mm; "
                        "rows_unexcused = rows that differ from the oracle's beyond 2e-3 mm + 4e-5 mm x "
                        "their crossing conditioning without an oracle near-face flag; each side on its "
                        "own trajectory (free-running)" % (s, args.mode))
    if rank == 0:
        print(json.dumps(out))
    ctx.close()
    if dist:
        dist.destroy_process_group()
    return 0


def exclusion_voxels(pct, cfg, hull_np, sub, sub_np, local, block):
    """The voxels the comparison rule leaves out for a history sample: the
    oracle's rows (with margins and crossing conditioning) against the GPU's
    rows of the same protons, block by block."""
    import oracle as O
    from oracle.compare import Exclusion
    geo = O.Geometry(cfg.shape, (cfg.voxel,) * 3, cfg.origin, mask=hull_np)
    rowptr, jo, lo, margin, cond = O.rows(geo, sub_np, with_cond=True)
    n = int(sub["wepl"].numel())
    ex = Exclusion(cfg.n_vox, block)
    with pct.Context(cfg.shape, cfg.voxel, cfg.origin, hull=hull_np, device=local) as c:
        c.load_histories(sub)
        for a in range(0, n, 8192):
            k = min(n, a + 8192) - a
            _, _, nnz = c.rows(a, k, max_nnz=0)
            W = max(int(nnz.max().item()), 1)
            idx, ln, nnz = c.rows(a, k, max_nnz=W)
            e0, e1 = int(rowptr[a]), int(rowptr[a + k])
            ex.add(a, idx.cpu().numpy(), ln.cpu().numpy(), nnz.cpu().numpy(), rowptr[a:a + k + 1] - e0,
                   jo[e0:e1], lo[e0:e1], margin[a:a + k], cond[a:a + k])
    return ex.finish()


def run_adam(args):
    """50 Adam steps on ||A x - b||^2 + 0.01 TV(x) (128x128x32 grid, 4e6 protons):
    each step = A x, A^T r (paths recomputed), TV and its gradient, one Adam update."""
    import numpy as np
    import torch

    import paper_1802_01070_b300 as pct
    import synth
    from paper_1802_01070_b300 import autograd as AG
    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", "0")))
    torch.cuda.set_device(dev)
    cfg = synth.CONFIGS["diff"]
    n = args.protons or cfg.n_protons
    if n != cfg.n_protons:
        cfg = synth.scaled(cfg, n)
    rsp, hull = synth.phantom(cfg)
    hist = synth.histories(cfg, dev, chunk=1 << 24, rsp=rsp)
    steps = 50
    with pct.Context(cfg.shape, cfg.voxel, cfg.origin, hull=hull.numpy(), device=dev.index) as ctx:
        ctx.load_histories(hist)
        b = hist["wepl"].clone()
        valid = int((ctx.hull_states()[:, 10] > 0.5).sum().item())
        x0 = torch.from_numpy(hull.numpy().astype(np.float32)).to(dev)
        for _ in range(max(args.warmup, 1)):
            AG.reconstruct_tv_adam(ctx, b, x0, steps=2, lr=1e-2)
        torch.cuda.synchronize(dev)
        ctx.reset_stats()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        clk = ClockSampler(_pci_id(torch, dev))
        clk.start()
        e0.record()
        # the reconstruction starts from the device-resident histories: the
        # per-proton records are computed once, inside the timed region
        ctx.load_histories(hist)
        x, losses = AG.reconstruct_tv_adam(ctx, b, x0, steps=steps, lr=1e-2)
        e1.record()
        torch.cuda.synchronize(dev)
        clocks = clk.stop()
        ms = e0.elapsed_time(e1)
        launches = int(ctx.stat(pct.PCT_STAT_LAUNCHES))
    per_step = ms / steps
    print(json.dumps({
        "metric": "TV-regularised Adam reconstruction: proton-rows/s per step (A x + A^T r)",
        "value": valid / (per_step * 1e-3), "unit": UNIT, "n_gpus": 1, "steps": steps,
        "warmup": max(args.warmup, 1), "ms_per_step": per_step, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": "diff: %dx%dx%d grid, %d protons over %d angles, loss ||Ax-b||^2 + "
                               "0.01 TV(x), %d Adam steps, lr 1e-2" % (*cfg.shape, n, cfg.n_angles, steps),
                   "rows_in_hull": valid},
        "loss_first": losses[0], "loss_last": losses[-1], "recon_s": ms * 1e-3,
        "gpu_launches": launches, "clocks": clocks}))
    return 0


def run_batch(args):
    """16 validation scans (1e5..2e6 protons, 64x64x8..128x128x32 grids): one
    batched persistent launch (graph-captured, autotuned CTA size) against the
    same scans solved one pct_solve after another."""
    import numpy as np
    import torch

    import paper_1802_01070_b300 as pct
    import synth
    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", "0")))
    torch.cuda.set_device(dev)
    cfgs = synth.validation_scans()
    ctxs, hulls, valid = [], [], 0
    for cfg in cfgs:
        rsp, hull = synth.phantom(cfg)
        hist = synth.histories(cfg, dev, chunk=1 << 24, rsp=rsp)
        c = pct.Context(cfg.shape, cfg.voxel, cfg.origin, hull=hull.numpy(), device=dev.index)
        c.load_histories(hist)
        valid += int((c.hull_states()[:, 10] > 0.5).sum().item())
        ctxs.append(c)
        hulls.append(torch.from_numpy(hull.numpy().astype(np.float32)).to(dev))
    c0 = ctxs[0]
    c0.set_option(pct.PCT_OPT_GRAPH, 1)
    c0.set_option(pct.PCT_OPT_AUTOTUNE, 1)
    iters = [c.iters for c in cfgs]
    lams = [c.lam for c in cfgs]
    blocks = [c.block for c in cfgs]

    def batched():
        xs = [h.clone() for h in hulls]
        pct.pct_solve_batch(ctxs, iters, lams, blocks, xs)
        return xs

    def sequential():
        xs = [h.clone() for h in hulls]
        for c, cfg, x in zip(ctxs, cfgs, xs):
            c.solve(x, cfg.iters, cfg.lam, cfg.block)
        return xs

    def timed(fn, reps):
        for _ in range(max(args.warmup, 1)):
            fn()
        c0.synchronize()
        torch.cuda.synchronize(dev)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            out = fn()
        e1.record()
        torch.cuda.synchronize(dev)
        c0.synchronize()
        return e0.elapsed_time(e1) / reps, out

    c0.reset_stats()
    clk = ClockSampler(_pci_id(torch, dev))
    clk.start()
    ms_b, xb = timed(batched, args.steps)
    clocks = clk.stop()
    launches = int(c0.stat(pct.PCT_STAT_LAUNCHES))
    ms_s, xsq = timed(sequential, args.steps)
    xsq2 = sequential()
    torch.cuda.synchronize(dev)
    seq_abs = max(float(torch.abs(a - b).max()) for a, b in zip(xsq2, xsq))
    worst_abs = max(float(torch.abs(a - b).max()) for a, b in zip(xb, xsq))
    worst = max(float((torch.abs(a - b) / torch.abs(b))[torch.abs(b) > 0.05].max()) for a, b in zip(xb, xsq))
    within = [((torch.abs(a - b) <= 1e-3 * torch.abs(b)) | (b == 0)).float() for a, b in zip(xb, xsq)]
    frac_within = float(sum(w.sum() for w in within) / sum(w.numel() for w in within))
    rows_iter = valid * cfgs[0].iters
    print(json.dumps({
        "metric": "batched validation scans: proton-rows/s per iteration (16 scans, one launch)",
        "value": rows_iter / (ms_b * 1e-3), "unit": UNIT, "n_gpus": 1, "steps": args.steps,
        "warmup": max(args.warmup, 1), "ms_per_step": ms_b, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": "16 scans, protons log-uniform 1e5..2e6 (total %d, %d cross the hull), "
                               "grids 64x64x8..128x128x32, 6 iterations, block 3200, graph-captured "
                               "cooperative launch" % (sum(c.n_protons for c in cfgs), valid),
                   "cta": c0.stat(pct.PCT_STAT_BATCH_CTA), "ctas": c0.stat(pct.PCT_STAT_BATCH_CTAS),
                   "lanes_per_proton": c0.stat(pct.PCT_STAT_BATCH_LANES),
                   "tuning": "CTA size x lanes per proton autotuned on the first call"},
        "sequential_ms_per_step": ms_s, "speedup_vs_sequential": ms_s / ms_b,
        "max_rel_diff_vs_sequential": worst, "max_abs_diff_vs_sequential": worst_abs,
        "max_abs_diff_sequential_vs_sequential": seq_abs,
        "frac_voxels_within_1e-3_vs_sequential": frac_within,
        "diff_note": "relative difference over voxels with |x| > 0.05; both runs use the same "
                     "kernels, only the order of FP32 atomics differs",
        "gpu_launches": launches, "clocks": clocks}))
    for c in ctxs:
        c.close()
    return 0


# ----------------------------------------------------------------------------
# Studies around the solve: block size, FBP start, cleaning, image regions
# ----------------------------------------------------------------------------

def _setup(args, outlier_frac=0.0):
    import numpy as np
    import torch

    import paper_1802_01070_b300 as pct
    import synth
    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", "0")))
    torch.cuda.set_device(dev)
    cfg = synth.CONFIGS[args.config]
    n = args.protons or cfg.n_protons
    if n != cfg.n_protons:
        cfg = synth.scaled(cfg, n)
    rsp, hull = synth.phantom(cfg)
    hist = synth.histories(cfg, dev, chunk=1 << 24, rsp=rsp, outlier_frac=outlier_frac)
    ctx = pct.Context(cfg.shape, cfg.voxel, cfg.origin, hull=hull.numpy(), device=dev.index)
    ctx.load_histories(hist)
    hm = torch.from_numpy(hull.numpy().astype(bool)).to(dev)
    truth = rsp.to(dev)
    return pct, cfg, dev, hist, ctx, hm, truth, hull.numpy()


def _quality(ctx, x, b, valid, hm, truth):
    """Relative residual ||A x - b|| / ||b|| over rows with a hull path, mean
    |x - truth| / truth over hull voxels, and the mean RSP of each true value
    (the paper's insert means) with its error in %."""
    import torch
    y = ctx.forward(x)
    r = float(torch.linalg.vector_norm((y - b)[valid]) / torch.linalg.vector_norm(b[valid]))
    xt, tt = x[hm], truth[hm]
    err = float((torch.abs(xt - tt) / tt).mean())
    inserts = {}
    for v in torch.unique(tt).tolist():
        m = tt == v
        mean = float(xt[m].mean())
        inserts["%.2f" % v] = {"mean": mean, "err_pct": 100.0 * (mean - v) / v, "voxels": int(m.sum())}
    return r, err, inserts


def run_blocks(args):
    """Block-size study (Sec. IV-B: larger blocks make an iteration faster but
    not necessarily more accurate): the torso scan solved from x0 = 1 with
    B = 3200, 32000 and 320000, per iteration its time and rows/s, the
    residual and the RSP error against the phantom; and the final RSP against
    the FP64 oracle on a bounded sample of the same scan."""
    import numpy as np
    import torch
    pct, cfg, dev, hist, ctx, hm, truth, hull_np = _setup(args)
    b = hist["wepl"]
    valid = ctx.hull_states()[:, 10] > 0.5
    n_valid = int(valid.sum())
    x0 = hm.float()
    out = {"metric": "block-size study: proton-rows/s per iteration and RSP error vs truth per iteration",
           "unit": UNIT, "config": {"workload": "%s: %d protons, lambda %g, fused rows" % (cfg.name, ctx.n, cfg.lam)},
           "blocks": {}}
    clk = ClockSampler(_pci_id(torch, dev))
    clk.start()
    for B in (3200, 32000, 320000):
        x = x0.clone()
        ctx.solve(x.clone(), 1, cfg.lam, B)      # warm-up: lists and kernels
        ctx.synchronize()
        curve = []
        t_total = 0.0
        for it in range(cfg.iters):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            ctx.solve(x, 1, cfg.lam, B)
            e1.record()
            torch.cuda.synchronize(dev)
            ms = e0.elapsed_time(e1)
            t_total += ms
            r, err, ins = _quality(ctx, x, b, valid, hm, truth)
            curve.append({"iter": it + 1, "ms": ms, "rows_per_s": n_valid / (ms * 1e-3), "elapsed_s": t_total * 1e-3,
                          "residual": r, "rsp_mean_abs_rel_err": err, "inserts": ins})
        out["blocks"][str(B)] = curve
    out["clocks"] = clk.stop()
    # against the FP64 oracle on the first protons of the scan
    s = min(args.cpu_sample, ctx.n)
    if s > 0 and not args.no_cpu_baseline:
        import oracle as O
        import synth
        from oracle.compare import solve_parity
        sub = {k: v[:s].clone() for k, v in hist.items()}
        sub_np = synth.to_numpy(sub)
        geo = O.Geometry(cfg.shape, (cfg.voxel,) * 3, cfg.origin, mask=hull_np)
        rowptr, j, ln, margin, cond = O.rows(geo, sub_np, with_cond=True)
        A = O.csr(rowptr, j, ln, geo.n_vox)
        res = {}
        with pct.Context(cfg.shape, cfg.voxel, cfg.origin, hull=hull_np, device=dev.index) as c2:
            c2.load_histories(sub)
            for B in (3200, 32000, 320000):
                xg = x0.clone()
                c2.solve(xg, cfg.iters, cfg.lam, B)
                c2.synchronize()
                xo = O.drop(A, sub_np["wepl"].astype(np.float64), cfg.iters, cfg.lam, B, hull_np.astype(np.float64))
                ex = exclusion_voxels(pct, cfg, hull_np, sub, sub_np, dev.index, B)
                res[str(B)] = solve_parity(xg.cpu().numpy(), xo, hull_np, ex)
        out["vs_oracle"] = {"sample": "first %d protons, %d iterations" % (s, cfg.iters), "by_block": res}
    print(json.dumps(out))
    ctx.close()
    return 0


def run_fbp(args):
    """FBP initial iterate (Sec. I): its time on the scan, and the DROP
    convergence from it against x0 = 1 inside the hull (residual and RSP error
    after each iteration; the iterations the FBP start needs to reach the
    x0 = 1 start's final residual)."""
    import torch

    import synth
    pct, cfg, dev, hist, ctx, hm, truth, hull_np = _setup(args)
    bins = synth.fbp_bins(cfg)
    b = hist["wepl"]
    valid = ctx.hull_states()[:, 10] > 0.5
    block = args.block or cfg.block
    for _ in range(max(args.warmup, 1)):
        x_fbp = ctx.fbp(**bins)
    torch.cuda.synchronize(dev)
    ts = []
    for _ in range(max(args.steps, 1)):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        x_fbp = ctx.fbp(**bins)
        e1.record()
        torch.cuda.synchronize(dev)
        ts.append(e0.elapsed_time(e1))
    fbp_ms = statistics.median(ts)
    curves, reach = {}, {}
    for lam in (cfg.lam, 0.1):
        for name, start in (("ones", hm.float()), ("fbp", x_fbp)):
            x = start.clone()
            r, err, ins = _quality(ctx, x, b, valid, hm, truth)
            curve = [{"iter": 0, "residual": r, "rsp_mean_abs_rel_err": err, "inserts": ins}]
            for it in range(cfg.iters):
                ctx.solve(x, 1, lam, block)
                r, err, ins = _quality(ctx, x, b, valid, hm, truth)
                curve.append({"iter": it + 1, "residual": r, "rsp_mean_abs_rel_err": err, "inserts": ins})
            curves["%s, lambda %g" % (name, lam)] = curve
        # iterations from the FBP start to within 0.1 % of the x0 = 1 start's
        # final residual
        target = curves["ones, lambda %g" % lam][-1]["residual"] * 1.001
        reach["lambda %g" % lam] = next((c["iter"] for c in curves["fbp, lambda %g" % lam]
                                         if c["residual"] <= target), None)
    print(json.dumps({
        "metric": "FBP initial iterate: ms per FBP and DROP iterations to the x0=1 start's final residual",
        "value": fbp_ms, "unit": "ms", "higher_is_better": False,
        "config": {"workload": "%s: %d protons, bins %s, DROP lambda %g block %d" % (
            cfg.name, ctx.n, bins, cfg.lam, block)},
        "fbp_protons_per_s": ctx.n / (fbp_ms * 1e-3),
        "iterations_from_fbp_to_ones_final_residual": reach, "curves": curves}))
    ctx.close()
    return 0


def run_clean(args):
    """Data cleaning (Sec. IV-A): statistical outlier removal on the scan with
    2 % planted outliers; ms per call, protons/s, and what it removed."""
    import torch

    import synth
    pct, cfg, dev, hist, ctx, hm, truth, hull_np = _setup(args, outlier_frac=0.02)
    bins = synth.clean_bins(cfg)
    planted = synth.outlier_mask(cfg, frac=0.02, device=dev)
    ts, kept = [], 0
    for k in range(max(args.warmup, 1) + max(args.steps, 1)):
        ctx.load_histories(hist)
        torch.cuda.synchronize(dev)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        kept, flags = ctx.clean(**bins, keep=True)
        e1.record()
        torch.cuda.synchronize(dev)
        if k >= max(args.warmup, 1):
            ts.append(e0.elapsed_time(e1))
    ms = statistics.median(ts)
    f = flags.bool()
    print(json.dumps({
        "metric": "data cleaning: protons/s", "value": cfg.n_protons / (ms * 1e-3), "unit": "protons/s",
        "ms_per_call": ms, "higher_is_better": True,
        "config": {"workload": "%s: %d protons with 2%% planted outliers, bins %s" % (cfg.name, cfg.n_protons, bins)},
        "kept": kept, "kept_frac": kept / cfg.n_protons,
        "planted_removed_frac": float((~f[planted]).float().mean()),
        "clean_kept_frac": float(f[~planted].float().mean())}))
    ctx.close()
    return 0


def run_regions(args):
    """The paper's Algorithm 1 on one GPU against the plain solve: time, protons
    per region, and the RSP error of each against the phantom."""
    import torch
    pct, cfg, dev, hist, ctx, hm, truth, hull_np = _setup(args)
    b = hist["wepl"]
    valid = ctx.hull_states()[:, 10] > 0.5
    block = args.block or cfg.block
    res = {}
    # overlap: the paper's three 2.5 mm slices on each side, 7.5 mm
    halo = int(math.ceil(7.5 / cfg.voxel))
    for name, regions in (("plain", 0), ("2 regions", 2), ("4 regions", 4)):
        times = []
        for k in range(2):
            x = hm.float()
            torch.cuda.synchronize(dev)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            if regions:
                counts = ctx.solve_regions(x, regions, halo, cfg.iters, cfg.lam, block)
            else:
                ctx.solve(x, cfg.iters, cfg.lam, block)
                counts = [int(valid.sum())]
            e1.record()
            torch.cuda.synchronize(dev)
            times.append(e0.elapsed_time(e1))
        r, err, ins = _quality(ctx, x, b, valid, hm, truth)
        res[name] = {"ms": times[-1], "protons_per_region": counts, "halo_slices": halo if regions else 0,
                     "residual": r, "rsp_mean_abs_rel_err": err, "inserts": ins}
        if regions:
            # protons that fit no region (both hull end points in one region's slices)
            res[name]["note"] = "a proton may belong to two regions, or to none"
    print(json.dumps({"metric": "image regions (Algorithm 1) on one GPU vs the plain solve",
                      "config": {"workload": "%s: %d protons, %d iterations, block %d" % (
                          cfg.name, ctx.n, cfg.iters, block)}, "results": res}))
    ctx.close()
    return 0


def main():
    args = _args()
    if args.impl == "reference":
        return run_reference(args)
    tasks = {"adam": run_adam, "batch": run_batch, "blocks": run_blocks, "fbp": run_fbp, "clean": run_clean,
             "regions": run_regions}
    return tasks.get(args.task, run_ours)(args)


if __name__ == "__main__":
    sys.exit(main())
