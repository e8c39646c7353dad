"""pct-b300: proton-CT RSP reconstruction on one NVIDIA B300.

Python binding of ``libpct`` (C ABI in ``include/pct.h``): argument marshalling
only.  Every step of the hot path -- hull entry, most likely path, voxel walk,
row dot products, DROP scatter and apply, A x, A^T y -- runs in the library's
CUDA kernels.  torch is used for device memory and streams.  There is no CPU
fallback: if ``libpct.so`` is missing the import of the native handle fails.

The module-level ``pct_*`` functions mirror the C entry points one to one;
``Context`` bundles them for convenience.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

__all__ = ["PctError", "Context", "load_library", "HIST_FIELDS", "STATE_FIELDS",
           "PCT_OPT_CTA_THREADS", "PCT_OPT_MLP_STEP_UM", "PCT_OPT_MEM_CAP_BYTES", "PCT_OPT_TIMING",
           "PCT_STAT_LAUNCHES", "PCT_STAT_FUSED_LAUNCHES", "PCT_STAT_FUSED_MS",
           "PCT_STAT_DEVICE_BYTES", "PCT_STAT_N_PROTONS", "PCT_STAT_N_HULL_VOXELS"]

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libpct.so")

PCT_OK, PCT_ERR_ARG, PCT_ERR_CUDA, PCT_ERR_OOM, PCT_ERR_STATE, PCT_ERR_TIMEOUT, PCT_ERR_DEVICE = range(7)
STATUS_NAMES = {0: "PCT_OK", 1: "PCT_ERR_ARG", 2: "PCT_ERR_CUDA", 3: "PCT_ERR_OOM",
                4: "PCT_ERR_STATE", 5: "PCT_ERR_TIMEOUT", 6: "PCT_ERR_DEVICE"}
PCT_OPT_CTA_THREADS, PCT_OPT_MLP_STEP_UM, PCT_OPT_MEM_CAP_BYTES, PCT_OPT_TIMING, PCT_OPT_MODE = 1, 2, 3, 4, 5
PCT_OPT_GRAPH, PCT_OPT_AUTOTUNE, PCT_OPT_SPIN_LIMIT, PCT_OPT_TEST_UNREACHABLE_BARRIER = 6, 7, 8, 9
PCT_STAT_BATCH_CTA, PCT_STAT_BATCH_CTAS, PCT_STAT_GRAPH_REPLAYS, PCT_STAT_TIMED_LAUNCHES = 9, 10, 11, 12
PCT_MODE_FUSED, PCT_MODE_CSR, PCT_MODE_PACKED = 0, 1, 2
PCT_OPT_CHORD_CODE, PCT_OPT_BATCH_LANES = 10, 11
PCT_STAT_BATCH_LANES = 13
PCT_OPT_WALK, PCT_WALK_LANES, PCT_WALK_ROUNDS = 12, 0, 1
PCT_STAT_WALK_FALLBACKS = 14
PCT_OPT_PERSISTENT_BLOCK = 13
PCT_OPT_SOLVE_GRAPH = 14
PCT_STAT_SOLVE_GRAPH_REPLAYS = 15
PCT_CHORD_FIXED16, PCT_CHORD_FP16 = 0, 1
(PCT_STAT_LAUNCHES, PCT_STAT_FUSED_LAUNCHES, PCT_STAT_FUSED_MS, PCT_STAT_DEVICE_BYTES,
 PCT_STAT_N_PROTONS, PCT_STAT_N_HULL_VOXELS, PCT_STAT_ROW_ENTRIES, PCT_STAT_ROW_BYTES) = 1, 2, 3, 4, 5, 6, 7, 8

HIST_FIELDS = ("in_x", "in_y", "in_z", "out_x", "out_y", "out_z",
               "theta_in", "psi_in", "theta_out", "psi_out", "phi", "wepl")
STATE_FIELDS = ("u_in", "u_out", "t0", "theta0", "v0", "psi0", "t2", "theta2", "v2", "psi2",
                "valid", "spare")

# every symbol include/pct.h declares
EXPORTS = ("pct_create", "pct_destroy", "pct_last_error", "pct_set_option", "pct_get_option",
           "pct_load_histories", "pct_hull_states", "pct_mlp", "pct_rows", "pct_forward",
           "pct_adjoint", "pct_solve", "pct_solve_host", "pct_synchronize", "pct_get_stat",
           "pct_reset_stats", "pct_solve_noalloc", "pct_build_rows", "pct_tv", "pct_adam",
           "pct_solve_batch", "pct_hull_distance", "pct_tan_angle", "pct_peak_fp32",
           "pct_peak_atomic", "pct_clean", "pct_fbp", "pct_solve_regions")


class PctError(RuntimeError):
    def __init__(self, status, message):
        super().__init__("%s: %s" % (STATUS_NAMES.get(status, status), message))
        self.status = status
        self.message = message


class pct_grid(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("nz", ctypes.c_int32),
                ("dx", ctypes.c_float), ("dy", ctypes.c_float), ("dz", ctypes.c_float),
                ("ox", ctypes.c_float), ("oy", ctypes.c_float), ("oz", ctypes.c_float)]


_lib = None


def load_library(path: str = LIB_PATH):
    """Load libpct.so (built in-tree by ``paper_1802_01070_b300.build``)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError("libpct.so is not built (%s); run paper_1802_01070_b300.build.build()" % path)
    lib = ctypes.CDLL(path)
    P, I32, I64, F = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_float
    sig = {
        "pct_create": ([P, P, P, ctypes.c_int, P], ctypes.c_int),
        "pct_destroy": ([P], None),
        "pct_last_error": ([P], ctypes.c_char_p),
        "pct_set_option": ([P, I32, I64], ctypes.c_int),
        "pct_get_option": ([P, I32, P], ctypes.c_int),
        "pct_load_histories": ([P, I64, P, P, P, P, P, P, ctypes.c_int], ctypes.c_int),
        "pct_hull_states": ([P, I64, I64, P], ctypes.c_int),
        "pct_hull_distance": ([P, P], ctypes.c_int),
        "pct_mlp": ([P, I64, I64, I32, P, P], ctypes.c_int),
        "pct_rows": ([P, I64, I64, I32, P, P, P], ctypes.c_int),
        "pct_forward": ([P, P, P], ctypes.c_int),
        "pct_adjoint": ([P, P, P], ctypes.c_int),
        "pct_solve": ([P, I32, F, I64, P], ctypes.c_int),
        "pct_solve_host": ([P, I32, F, I64, P], ctypes.c_int),
        "pct_synchronize": ([P], ctypes.c_int),
        "pct_get_stat": ([P, I32, P], ctypes.c_int),
        "pct_reset_stats": ([P], ctypes.c_int),
        "pct_build_rows": ([P], ctypes.c_int),
        "pct_solve_batch": ([P, I32, P, P, P, P], ctypes.c_int),
        "pct_tv": ([P, P, F, P, P], ctypes.c_int),
        "pct_adam": ([P, P, P, P, P, I64, F, F, F, F, I32], ctypes.c_int),
        "pct_solve_noalloc": ([P, P, I64, P, P, P, P, P, P, I32, F, I64, P, ctypes.c_int, P],
                              ctypes.c_int),
        "pct_tan_angle": ([P, P, I64, P], ctypes.c_int),
        "pct_peak_fp32": ([ctypes.c_int, I32, P, P], ctypes.c_int),
        "pct_peak_atomic": ([ctypes.c_int, I64, I32, P, P], ctypes.c_int),
        "pct_clean": ([P, P, P, P], ctypes.c_int),
        "pct_fbp": ([P, P, P, P], ctypes.c_int),
        "pct_solve_regions": ([P, I32, I32, I32, F, I64, P, P], ctypes.c_int),
    }
    for name, (args, res) in sig.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = res
    _lib = lib
    return lib


def _check(ctx, status):
    if status != PCT_OK:
        msg = load_library().pct_last_error(ctx)
        raise PctError(status, msg.decode() if msg else "")


def _dptr(t, dtype, n=None, what="tensor"):
    """Device pointer of a contiguous CUDA tensor of the given dtype (and size)."""
    import torch
    if not (torch.is_tensor(t) and t.is_cuda):
        raise TypeError("%s must be a CUDA tensor" % what)
    if t.dtype != dtype or not t.is_contiguous():
        raise TypeError("%s must be a contiguous %s tensor" % (what, dtype))
    if n is not None and t.numel() < n:
        raise ValueError("%s has %d elements, needs %d" % (what, t.numel(), n))
    return ctypes.c_void_p(t.data_ptr())


# ----------------------------------------------------------------------------
# One-to-one wrappers of the C entry points (handles are ctypes.c_void_p).
# ----------------------------------------------------------------------------

def pct_create(shape, voxel, origin, hull_mask=None, device=0, stream=None):
    lib = load_library()
    g = pct_grid(int(shape[0]), int(shape[1]), int(shape[2]), float(voxel[0]), float(voxel[1]),
                 float(voxel[2]), float(origin[0]), float(origin[1]), float(origin[2]))
    keep = None
    mp = None
    if hull_mask is not None:
        keep = np.ascontiguousarray(np.asarray(hull_mask, dtype=np.uint8).reshape(-1))
        if keep.size != int(shape[0]) * int(shape[1]) * int(shape[2]):
            raise ValueError("hull mask size does not match the grid")
        mp = keep.ctypes.data
    h = ctypes.c_void_p()
    st = lib.pct_create(ctypes.byref(h), ctypes.byref(g), mp, int(device),
                        ctypes.c_void_p(stream) if stream else None)
    if st != PCT_OK:
        raise PctError(st, lib.pct_last_error(None).decode())
    return h


def pct_destroy(ctx):
    load_library().pct_destroy(ctx)


def pct_set_option(ctx, key, value):
    _check(ctx, load_library().pct_set_option(ctx, int(key), int(value)))


def pct_get_option(ctx, key):
    v = ctypes.c_int64()
    _check(ctx, load_library().pct_get_option(ctx, int(key), ctypes.byref(v)))
    return v.value


def pct_load_histories(ctx, hist):
    """hist: dict of 12 equal-length float32 arrays (CUDA tensors, or host arrays)."""
    import torch
    cols = [hist[k] for k in HIST_FIELDS]
    on_dev = all(torch.is_tensor(c) and c.is_cuda for c in cols)
    keep = []
    ptrs = []
    n = None
    for k, c in zip(HIST_FIELDS, cols):
        if on_dev:
            p = _dptr(c, torch.float32, what=k)
            m = c.numel()
        else:
            if torch.is_tensor(c):
                a = c.detach().cpu().to(torch.float32).contiguous()
            else:
                a = np.ascontiguousarray(np.asarray(c, dtype=np.float32))
            keep.append(a)
            p = ctypes.c_void_p(a.data_ptr() if torch.is_tensor(a) else a.ctypes.data)
            m = a.numel() if torch.is_tensor(a) else a.size
        if n is None:
            n = m
        elif m != n:
            raise ValueError("history arrays differ in length")
        ptrs.append(p)
    A3 = ctypes.c_void_p * 3
    A2 = ctypes.c_void_p * 2
    st = load_library().pct_load_histories(
        ctx, int(n), A3(*ptrs[0:3]), A3(*ptrs[3:6]), A2(ptrs[6], ptrs[7]), A2(ptrs[8], ptrs[9]),
        ptrs[10], ptrs[11], 1 if on_dev else 0)
    _check(ctx, st)
    return int(n)


def pct_hull_states(ctx, first, count, out):
    import torch
    _check(ctx, load_library().pct_hull_states(ctx, int(first), int(count),
                                               _dptr(out, torch.float32, 12 * count, "out")))


def pct_hull_distance(ctx, n_vox, out):
    import torch
    _check(ctx, load_library().pct_hull_distance(ctx, _dptr(out, torch.uint8, n_vox, "out")))


def pct_mlp(ctx, first, count, max_pts, out_xyz, out_npts):
    import torch
    _check(ctx, load_library().pct_mlp(ctx, int(first), int(count), int(max_pts),
                                       _dptr(out_xyz, torch.float32, 3 * max_pts * count, "out_xyz"),
                                       _dptr(out_npts, torch.int32, count, "out_npts")))


def pct_rows(ctx, first, count, max_nnz, out_idx, out_len, out_nnz):
    import torch
    _check(ctx, load_library().pct_rows(ctx, int(first), int(count), int(max_nnz),
                                        _dptr(out_idx, torch.int32, max_nnz * count, "out_idx"),
                                        _dptr(out_len, torch.float32, max_nnz * count, "out_len"),
                                        _dptr(out_nnz, torch.int32, count, "out_nnz")))


def pct_forward(ctx, x, y):
    import torch
    _check(ctx, load_library().pct_forward(ctx, _dptr(x, torch.float32, what="x"),
                                           _dptr(y, torch.float32, what="y")))


def pct_adjoint(ctx, y, g):
    import torch
    _check(ctx, load_library().pct_adjoint(ctx, _dptr(y, torch.float32, what="y"),
                                           _dptr(g, torch.float32, what="g")))


def pct_solve(ctx, iters, lam, block_size, x):
    import torch
    _check(ctx, load_library().pct_solve(ctx, int(iters), float(lam), int(block_size),
                                         _dptr(x, torch.float32, what="x")))


def pct_solve_host(ctx, iters, lam, block_size, x_host):
    """x_host: contiguous float32 numpy array or CPU tensor, updated in place."""
    import torch
    if torch.is_tensor(x_host):
        if x_host.is_cuda or x_host.dtype != torch.float32 or not x_host.is_contiguous():
            raise TypeError("x_host must be a contiguous float32 CPU tensor")
        p = ctypes.c_void_p(x_host.data_ptr())
    else:
        if x_host.dtype != np.float32 or not x_host.flags.c_contiguous:
            raise TypeError("x_host must be a contiguous float32 array")
        p = ctypes.c_void_p(x_host.ctypes.data)
    _check(ctx, load_library().pct_solve_host(ctx, int(iters), float(lam), int(block_size), p))


PCT_NOALLOC_MAX_PROTONS = 65536
PCT_NOALLOC_MAX_VOXELS = 1048576


def pct_solve_noalloc(shape, voxel, origin, hull_mask, hist, iters, lam, block_size, x,
                      device=None, stream=None):
    """DROP reconstruction that allocates no device memory (see include/pct.h).

    hull_mask: CUDA uint8 tensor of nx*ny*nz bytes; hist: dict of 12 CUDA float32
    tensors of equal length; x: CUDA float32 tensor (n voxels), updated in place.
    Every tensor must be on one device, which the call runs on (``device``, if
    given, must name it).  Returns the C status (0 = PCT_OK) instead of raising,
    so callers can test limits.
    """
    import torch
    g = pct_grid(int(shape[0]), int(shape[1]), int(shape[2]), float(voxel[0]), float(voxel[1]),
                 float(voxel[2]), float(origin[0]), float(origin[1]), float(origin[2]))
    n_vox = int(shape[0]) * int(shape[1]) * int(shape[2])
    cols = [hist[k] for k in HIST_FIELDS]
    n = cols[0].numel()
    ptrs = [_dptr(c, torch.float32, n, k) for k, c in zip(HIST_FIELDS, cols)]
    xp = _dptr(x, torch.float32, n_vox, "x")
    mp = _dptr(hull_mask, torch.uint8, n_vox, "hull_mask")
    dev = x.device.index if x.device.index is not None else torch.cuda.current_device()
    if device is not None and int(device) != dev:
        raise ValueError("x is on cuda:%d, device=%d was given" % (dev, int(device)))
    for name, t in [("hull_mask", hull_mask)] + list(zip(HIST_FIELDS, cols)):
        if t.device != x.device:
            raise ValueError("%s is on %s, x on %s" % (name, t.device, x.device))
    A3 = ctypes.c_void_p * 3
    A2 = ctypes.c_void_p * 2
    h = int(stream.cuda_stream) if stream is not None else int(torch.cuda.current_stream(dev).cuda_stream)
    return load_library().pct_solve_noalloc(
        ctypes.byref(g), mp, int(n), A3(*ptrs[0:3]),
        A3(*ptrs[3:6]), A2(ptrs[6], ptrs[7]), A2(ptrs[8], ptrs[9]), ptrs[10], ptrs[11], int(iters),
        float(lam), int(block_size), xp, int(dev),
        ctypes.c_void_p(h) if h else None)


def pct_tan_angle(t, out):
    """out = the record kernel's FP64 tangent of the angles t (CUDA float64 tensors)."""
    import torch
    n = t.numel()
    h = int(torch.cuda.current_stream(t.device).cuda_stream)
    st = load_library().pct_tan_angle(_dptr(t, torch.float64, what="t"), _dptr(out, torch.float64, n, "out"),
                                      int(n), ctypes.c_void_p(h) if h else None)
    if st != PCT_OK:
        raise PctError(st, "pct_tan_angle")


def pct_peak_fp32(device=0, repeats=5):
    """(TFLOP/s, best ms) of the library's FP32 FMA microbenchmark on ``device``."""
    t, ms = ctypes.c_double(), ctypes.c_double()
    st = load_library().pct_peak_fp32(int(device), int(repeats), ctypes.byref(t), ctypes.byref(ms))
    if st != PCT_OK:
        raise PctError(st, "pct_peak_fp32")
    return t.value, ms.value


def pct_peak_atomic(n_slots, device=0, repeats=5):
    """(1e9 float2 atomics/s, best ms) to random slots of an n_slots float2 array."""
    g, ms = ctypes.c_double(), ctypes.c_double()
    st = load_library().pct_peak_atomic(int(device), int(n_slots), int(repeats), ctypes.byref(g),
                                        ctypes.byref(ms))
    if st != PCT_OK:
        raise PctError(st, "pct_peak_atomic")
    return g.value, ms.value


def pct_tv(ctx, x, eps, grad, value):
    import torch
    _check(ctx, load_library().pct_tv(ctx, _dptr(x, torch.float32, what="x"), float(eps),
                                      _dptr(grad, torch.float32, what="grad"),
                                      _dptr(value, torch.float64, 1, "value")))


def pct_adam(ctx, x, grad, m, v, lr, beta1, beta2, eps, step):
    import torch
    n = x.numel()
    _check(ctx, load_library().pct_adam(ctx, _dptr(x, torch.float32, what="x"),
                                        _dptr(grad, torch.float32, n, "grad"),
                                        _dptr(m, torch.float32, n, "m"), _dptr(v, torch.float32, n, "v"),
                                        int(n), float(lr), float(beta1), float(beta2), float(eps),
                                        int(step)))


def pct_solve_batch(contexts, iters, lams, blocks, xs):
    """Batched DROP over several Contexts (one scan each), in one persistent launch.

    contexts: list of Context; iters, lams, blocks: per-scan lists; xs: list of
    CUDA float32 tensors, updated in place.  Ordered on the first context's stream.
    """
    import torch
    k = len(contexts)
    if not (len(iters) == len(lams) == len(blocks) == len(xs) == k) or k == 0:
        raise ValueError("one iters, lambda, block and x per context")
    H = (ctypes.c_void_p * k)(*[c.handle for c in contexts])
    IT = (ctypes.c_int32 * k)(*[int(v) for v in iters])
    LA = (ctypes.c_float * k)(*[float(v) for v in lams])
    BL = (ctypes.c_int64 * k)(*[int(v) for v in blocks])
    X = (ctypes.c_void_p * k)(*[_dptr(x, torch.float32, c.n_vox, "x").value for c, x in zip(contexts, xs)])
    with _Ordered(contexts[0]):
        _check(contexts[0].handle, load_library().pct_solve_batch(H, k, IT, LA, BL, X))


class pct_clean_params(ctypes.Structure):
    _fields_ = [("n_angle", ctypes.c_int32), ("n_t", ctypes.c_int32), ("n_v", ctypes.c_int32),
                ("angle_step", ctypes.c_double), ("t_min", ctypes.c_double), ("dt", ctypes.c_double),
                ("v_min", ctypes.c_double), ("dv", ctypes.c_double), ("k_sigma", ctypes.c_double)]


def pct_clean(ctx, n_angle, angle_step, n_t, t_min, dt, n_v, v_min, dv, k_sigma=3.0, keep_out=None):
    """Statistical outlier removal of the loaded histories; returns the kept count.
    keep_out: optional CUDA uint8 tensor of n bytes (1 = kept)."""
    import torch
    prm = pct_clean_params(int(n_angle), int(n_t), int(n_v), float(angle_step), float(t_min), float(dt),
                           float(v_min), float(dv), float(k_sigma))
    kp = _dptr(keep_out, torch.uint8, what="keep_out") if keep_out is not None else None
    nk = ctypes.c_int64()
    _check(ctx, load_library().pct_clean(ctx, ctypes.byref(prm), kp, ctypes.byref(nk)))
    return nk.value


class pct_fbp_params(ctypes.Structure):
    _fields_ = [("n_angle", ctypes.c_int32), ("n_t", ctypes.c_int32), ("n_v", ctypes.c_int32),
                ("angle_step", ctypes.c_double), ("t_min", ctypes.c_double), ("dt", ctypes.c_double),
                ("v_min", ctypes.c_double), ("dv", ctypes.c_double)]


def pct_fbp(ctx, n_vox, n_angle, angle_step, n_t, t_min, dt, n_v, v_min, dv, x, sino_out=None):
    """FBP image of the loaded histories into the CUDA float32 tensor x (n voxels);
    sino_out: optional CUDA float32 tensor of n_angle * n_v * n_t (filtered sinogram)."""
    import torch
    prm = pct_fbp_params(int(n_angle), int(n_t), int(n_v), float(angle_step), float(t_min), float(dt),
                         float(v_min), float(dv))
    sp = None
    if sino_out is not None:
        sp = _dptr(sino_out, torch.float32, int(n_angle) * int(n_v) * int(n_t), "sino_out")
    _check(ctx, load_library().pct_fbp(ctx, ctypes.byref(prm), _dptr(x, torch.float32, n_vox, "x"), sp))


def pct_build_rows(ctx):
    _check(ctx, load_library().pct_build_rows(ctx))


def pct_synchronize(ctx):
    _check(ctx, load_library().pct_synchronize(ctx))


def pct_get_stat(ctx, key):
    v = ctypes.c_double()
    _check(ctx, load_library().pct_get_stat(ctx, int(key), ctypes.byref(v)))
    return v.value


def pct_reset_stats(ctx):
    _check(ctx, load_library().pct_reset_stats(ctx))


# ----------------------------------------------------------------------------
# Convenience object
# ----------------------------------------------------------------------------

CUDA_STREAM_LEGACY = 1   # cudaStreamLegacy: the legacy default stream


def _stream_handle(stream):
    """C handle of a torch stream; torch's default stream is the legacy default stream."""
    h = int(stream.cuda_stream)
    return h if h else CUDA_STREAM_LEGACY


class _Ordered:
    """Orders library work on the context stream after, and before, work on the
    caller's current torch stream (no-op when they are the same stream)."""

    def __init__(self, ctx):
        self.ctx = ctx

    def __enter__(self):
        import torch
        self.cur = torch.cuda.current_stream(self.ctx.device)
        if self.cur != self.ctx.stream:
            self.ctx.stream.wait_stream(self.cur)
        return self

    def __exit__(self, *a):
        if self.cur != self.ctx.stream:
            self.cur.wait_stream(self.ctx.stream)


class Context:
    """One reconstruction grid + hull on one GPU, with its loaded protons.

    ``stream``: the torch.cuda.Stream the library enqueues on (default: the
    current stream of ``device`` at creation).  Every method orders its library
    work after the caller's current torch stream and makes that stream wait for
    it, so tensors can be used from torch right away.
    """

    def __init__(self, shape, voxel, origin, hull=None, device=0, stream=None):
        import torch
        if np.isscalar(voxel):
            voxel = (voxel, voxel, voxel)
        self.shape = tuple(int(v) for v in shape)
        self.n_vox = self.shape[0] * self.shape[1] * self.shape[2]
        self.device = torch.device("cuda", device)
        if stream is None:
            stream = torch.cuda.current_stream(self.device)
        self.stream = stream
        if torch.is_tensor(hull):
            hull = hull.detach().cpu().numpy()
        self._h = pct_create(self.shape, voxel, origin, hull, device, _stream_handle(stream))
        self.n = 0

    def close(self):
        if self._h is not None and self._h.value:
            pct_destroy(self._h)
        self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    @property
    def handle(self):
        return self._h

    def set_option(self, key, value):
        pct_set_option(self._h, key, value)

    def get_option(self, key):
        return pct_get_option(self._h, key)

    def load_histories(self, hist):
        with _Ordered(self):
            self.n = pct_load_histories(self._h, hist)
        return self.n

    def hull_states(self, first=0, count=None):
        import torch
        count = self.n - first if count is None else count
        out = torch.empty(count * 12 + 1, dtype=torch.float32, device=self.device)
        with _Ordered(self):
            pct_hull_states(self._h, first, count, out)
        return out[:count * 12].view(count, 12)

    def hull_distance(self):
        """Chessboard distance of every voxel to the hull (uint8, nz x ny x nx)."""
        import torch
        out = torch.empty(self.n_vox, dtype=torch.uint8, device=self.device)
        with _Ordered(self):
            pct_hull_distance(self._h, self.n_vox, out)
        return out.view(self.shape[2], self.shape[1], self.shape[0])

    def mlp(self, first=0, count=None, max_pts=512):
        import torch
        count = self.n - first if count is None else count
        pts = torch.zeros(count * max_pts * 3 + 1, dtype=torch.float32, device=self.device)
        npts = torch.zeros(count + 1, dtype=torch.int32, device=self.device)
        with _Ordered(self):
            pct_mlp(self._h, first, count, max_pts, pts, npts)
        return pts[:count * max_pts * 3].view(count, max_pts, 3), npts[:count]

    def rows(self, first=0, count=None, max_nnz=1024):
        import torch
        count = self.n - first if count is None else count
        idx = torch.zeros(count * max_nnz + 1, dtype=torch.int32, device=self.device)
        ln = torch.zeros(count * max_nnz + 1, dtype=torch.float32, device=self.device)
        nnz = torch.zeros(count + 1, dtype=torch.int32, device=self.device)
        with _Ordered(self):
            pct_rows(self._h, first, count, max_nnz, idx, ln, nnz)
        return (idx[:count * max_nnz].view(count, max_nnz), ln[:count * max_nnz].view(count, max_nnz),
                nnz[:count])

    def forward(self, x, out=None):
        import torch
        y = torch.empty(max(self.n, 1), dtype=torch.float32, device=self.device) if out is None else out
        _dptr(x, torch.float32, self.n_vox, "x")
        _dptr(y, torch.float32, self.n, "y")
        with _Ordered(self):
            pct_forward(self._h, x, y)
        return y[:self.n]

    def adjoint(self, y, out=None):
        import torch
        g = torch.empty(self.n_vox, dtype=torch.float32, device=self.device) if out is None else out
        if self.n == 0:
            y = torch.zeros(1, dtype=torch.float32, device=self.device)
        _dptr(y, torch.float32, self.n, "y")
        _dptr(g, torch.float32, self.n_vox, "g")
        with _Ordered(self):
            pct_adjoint(self._h, y, g)
        return g

    def solve(self, x, iters, lam, block_size):
        """DROP in place on the CUDA float32 tensor x (n voxels); returns x."""
        import torch
        _dptr(x, torch.float32, self.n_vox, "x")
        with _Ordered(self):
            pct_solve(self._h, iters, lam, block_size, x)
        return x

    def solve_host(self, x_host, iters, lam, block_size):
        if len(x_host) < self.n_vox:
            raise ValueError("x_host has fewer than n voxels")
        with _Ordered(self):
            pct_solve_host(self._h, iters, lam, block_size, x_host)
        return x_host

    def tv(self, x, eps=1e-6, grad=None):
        """(value as a 0-d float64 tensor, gradient) of the isotropic TV of x."""
        import torch
        g = torch.empty(self.n_vox, dtype=torch.float32, device=self.device) if grad is None else grad
        val = torch.empty(1, dtype=torch.float64, device=self.device)
        _dptr(x, torch.float32, self.n_vox, "x")
        _dptr(g, torch.float32, self.n_vox, "grad")
        with _Ordered(self):
            pct_tv(self._h, x, eps, g, val)
        return val[0], g

    def adam(self, x, grad, m, v, step, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8):
        with _Ordered(self):
            pct_adam(self._h, x, grad, m, v, lr, beta1, beta2, eps, step)

    def clean(self, n_angle, angle_step, n_t, t_min, dt, n_v, v_min, dv, k_sigma=3.0, keep=False):
        """Remove statistical outliers from the loaded protons (see pct_clean);
        returns the kept count, and the per-proton keep flags (CUDA uint8) when
        ``keep``."""
        import torch
        flags = torch.empty(max(self.n, 1), dtype=torch.uint8, device=self.device) if keep else None
        with _Ordered(self):
            kept = pct_clean(self._h, n_angle, angle_step, n_t, t_min, dt, n_v, v_min, dv, k_sigma, flags)
        old = self.n
        self.n = kept
        return (kept, flags[:old]) if keep else kept

    def solve_regions(self, x, n_regions, halo, iters, lam, block_size):
        """Algorithm 1 on one GPU (see pct_solve_regions) in place on x; returns
        the protons of each region."""
        import torch
        _dptr(x, torch.float32, self.n_vox, "x")
        cnt = (ctypes.c_int64 * int(n_regions))()
        with _Ordered(self):
            _check(self._h, load_library().pct_solve_regions(self._h, int(n_regions), int(halo), int(iters),
                                                              float(lam), int(block_size),
                                                              ctypes.c_void_p(x.data_ptr()), cnt))
        return list(cnt)

    def fbp(self, n_angle, angle_step, n_t, t_min, dt, n_v, v_min, dv, out=None, sinogram=False):
        """FBP initial iterate (CUDA float32, n voxels; 0 outside the hull), and
        the filtered sinogram (n_angle, n_v, n_t) when ``sinogram``."""
        import torch
        x = torch.empty(self.n_vox, dtype=torch.float32, device=self.device) if out is None else out
        q = torch.empty(int(n_angle) * int(n_v) * int(n_t), dtype=torch.float32,
                        device=self.device) if sinogram else None
        with _Ordered(self):
            pct_fbp(self._h, self.n_vox, n_angle, angle_step, n_t, t_min, dt, n_v, v_min, dv, x, q)
        return (x, q.view(int(n_angle), int(n_v), int(n_t))) if sinogram else x

    def build_rows(self):
        with _Ordered(self):
            pct_build_rows(self._h)

    def synchronize(self):
        pct_synchronize(self._h)

    def stat(self, key):
        return pct_get_stat(self._h, key)

    def reset_stats(self):
        pct_reset_stats(self._h)
