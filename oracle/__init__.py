"""FP64 CPU oracle for the proton-CT hot path -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline / reference
legs of ``bench.py`` may import this package.  The product library
(``paper_1802_01070_b300``) never imports, links or runs anything here, and
nothing here imports the product library.

The arithmetic lives in ``pct_oracle.c`` (plain C, FP64, OpenMP over protons
or over the rows of one DROP block); this module only marshals numpy arrays.
What each function follows (arXiv:1802.01070 prints neither formula):

* ``sigma`` / ``mlp_point`` / ``mlp_points`` -- the most likely path of
  Sec. I (cited there to Schulte et al. 2008): scattering matrices and the
  information-form MLP state.
* ``prepare`` -- hull entry and exit of the straight tracker lines (a reading:
  the paper names no hull rule).
* ``rows`` / ``csr`` -- the path data of A (Sec. I): chord length of the MLP
  polyline in each hull voxel it crosses.
* ``drop`` -- the DROP block-iterative update (Sec. IV-B).
* ``forward`` / ``adjoint`` -- A x and A^T y by a library sparse product.
* ``tv`` -- isotropic total variation with forward differences.

Parity status: pinned by ``tests/test_oracle_pins.py``; the whole
reconstruction is parity unpinned against the paper (no printed data).
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "pct_oracle.c")
_SO = os.path.join(_HERE, "liboracle.so")

HIST_FIELDS = ("in_x", "in_y", "in_z", "out_x", "out_y", "out_z",
               "theta_in", "psi_in", "theta_out", "psi_out", "phi", "wepl")

# 1/(beta^2 p^2) of a 200 MeV proton in water as a polynomial in depth (cm),
# MeV^-2 (the fit used with the Schulte et al. 2008 MLP).
COEF_200MEV_WATER = (7.457e-6, 4.548e-7, -5.777e-8, 1.301e-8, -9.228e-10, 2.687e-11)


def build(force: bool = False) -> str:
    """Compile pct_oracle.c into liboracle.so next to it (gcc, -O2, OpenMP)."""
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _SO)
    return _SO


class _Cfg(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("nz", ctypes.c_int32),
                ("highland", ctypes.c_int32),
                ("dx", ctypes.c_double), ("dy", ctypes.c_double), ("dz", ctypes.c_double),
                ("ox", ctypes.c_double), ("oy", ctypes.c_double), ("oz", ctypes.c_double),
                ("du", ctypes.c_double), ("dend", ctypes.c_double),
                ("coef", ctypes.c_double * 6)]


_lib = None


def _L():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_SO)
        P = ctypes.c_void_p
        lib.o_sigma.argtypes = [P, ctypes.c_double, ctypes.c_double, P]
        lib.o_mlp_point.argtypes = [P, P, P, ctypes.c_double, ctypes.c_double, P]
        lib.o_hull_entry.argtypes = [P, P, P, P, ctypes.c_double, P, P, P]
        lib.o_prepare.argtypes = [P, P, ctypes.c_int64, P, P, P, P]
        lib.o_mlp_points.argtypes = [P, P, ctypes.c_int64, P, ctypes.c_int32, P, P]
        lib.o_rows.argtypes = [P, P, ctypes.c_int64, P, P, P, P, P, P]
        lib.o_walk.argtypes = [P, P, ctypes.c_int64, P, P, P, ctypes.c_int64, P]
        lib.o_walk.restype = ctypes.c_int64
        lib.o_drop.argtypes = [ctypes.c_int64, ctypes.c_int64, P, P, P, P, ctypes.c_int32,
                               ctypes.c_double, ctypes.c_int64, P]
        lib.o_num_threads.restype = ctypes.c_int
        _lib = lib
    return _lib


def num_threads() -> int:
    """OpenMP threads the oracle's parallel loops use."""
    return int(_L().o_num_threads())


class Geometry:
    """Grid, hull mask and MLP options for the oracle.

    ``shape`` is (nx, ny, nz); voxel (ix, iy, iz) spans [o + i d, o + (i+1) d)
    per axis and has linear index j = ix + nx (iy + ny iz).  ``mask`` is a
    uint8 array of nx*ny*nz bytes in that order (None: every voxel is hull).
    ``du`` is the MLP sample spacing (mm, default the smallest voxel edge);
    no interior sample is taken within ``dend`` (default 1e-3 du) of the exit.
    """

    def __init__(self, shape, voxel, origin, mask=None, du=None, dend=None,
                 coef=COEF_200MEV_WATER, highland=True):
        self.shape = tuple(int(v) for v in shape)
        self.voxel = tuple(float(v) for v in voxel)
        self.origin = tuple(float(v) for v in origin)
        self.du = float(min(self.voxel) if du is None else du)
        self.dend = float(1e-3 * self.du if dend is None else dend)
        self.coef = tuple(float(c) for c in coef)
        self.highland = bool(highland)
        n = self.shape[0] * self.shape[1] * self.shape[2]
        self.n_vox = n
        if mask is None:
            self.mask = None
        else:
            m = np.ascontiguousarray(np.asarray(mask, dtype=np.uint8).reshape(-1))
            if m.size != n:
                raise ValueError("mask has %d bytes, grid has %d voxels" % (m.size, n))
            self.mask = m
        c = _Cfg()
        c.nx, c.ny, c.nz = self.shape
        c.highland = 1 if self.highland else 0
        c.dx, c.dy, c.dz = self.voxel
        c.ox, c.oy, c.oz = self.origin
        c.du = self.du
        c.dend = self.dend
        for k in range(6):
            c.coef[k] = self.coef[k]
        self._c = c

    def _cp(self):
        return ctypes.byref(self._c)

    def _mp(self):
        return None if self.mask is None else self.mask.ctypes.data


def _ptr(a):
    return a.ctypes.data


def _hist_arrays(hist):
    """(keep-alive list, ctypes array of 12 double pointers) for a history set."""
    cols = [np.ascontiguousarray(np.asarray(hist[k], dtype=np.float64)) for k in HIST_FIELDS]
    n = cols[0].size
    for c in cols:
        if c.size != n:
            raise ValueError("history arrays differ in length")
    arr = (ctypes.c_void_p * 12)(*[c.ctypes.data for c in cols])
    return cols, arr, n


def sigma(geo: Geometry, ua: float, ub: float) -> np.ndarray:
    """[int (ub-u)^2 f, int (ub-u) f, int f] times the Highland prefactor (cm, rad)."""
    out = np.zeros(3)
    _L().o_sigma(geo._cp(), float(ua), float(ub), _ptr(out))
    return out


def mlp_point(geo: Geometry, y0, y2, L: float, u1: float) -> np.ndarray:
    """MLP state (t cm, theta rad) at depth u1 from y0 at 0 and y2 at L (cm)."""
    a = np.ascontiguousarray(y0, dtype=np.float64)
    b = np.ascontiguousarray(y2, dtype=np.float64)
    out = np.zeros(2)
    if _L().o_mlp_point(geo._cp(), _ptr(a), _ptr(b), float(L), float(u1), _ptr(out)) != 0:
        raise FloatingPointError("singular scattering matrix")
    return out


def hull_entry(geo: Geometry, T, D, S: float, with_cond: bool = False):
    """(hit, s_hit, margin) for the line T + s D, s in [0, S]; with ``with_cond``
    also the conditioning of the crossing into the hit voxel (the line's length
    per unit of travel across the crossed face; 1 if it starts inside)."""
    t = np.ascontiguousarray(T, dtype=np.float64)
    d = np.ascontiguousarray(D, dtype=np.float64)
    s = np.zeros(1)
    m = np.full(1, np.inf)
    c = np.ones(1)
    hit = _L().o_hull_entry(geo._cp(), geo._mp(), _ptr(t), _ptr(d), float(S), _ptr(s), _ptr(m), _ptr(c))
    if with_cond:
        return bool(hit), float(s[0]), float(m[0]), float(c[0])
    return bool(hit), float(s[0]), float(m[0])


STATE_FIELDS = ("u_in", "u_out", "t0", "theta0", "v0", "psi0", "t2", "theta2", "v2", "psi2",
                "cos_phi", "sin_phi")


def prepare(geo: Geometry, hist):
    """Hull-frame state of every proton: (states (n, 12), valid (n,), margin (n,))."""
    keep, arr, n = _hist_arrays(hist)
    st = np.zeros((n, 12))
    valid = np.zeros(n, dtype=np.int32)
    margin = np.zeros(n)
    _L().o_prepare(geo._cp(), geo._mp(), n, arr, _ptr(st), _ptr(valid), _ptr(margin))
    del keep
    return st, valid.astype(bool), margin


def mlp_points(geo: Geometry, hist, max_pts: int):
    """MLP polyline per proton in lab mm: (pts (n, max_pts, 3), npts (n,))."""
    keep, arr, n = _hist_arrays(hist)
    pts = np.zeros((n, max_pts, 3))
    npts = np.zeros(n, dtype=np.int32)
    _L().o_mlp_points(geo._cp(), geo._mp(), n, arr, int(max_pts), _ptr(pts), _ptr(npts))
    del keep
    return pts, npts


def rows(geo: Geometry, hist, with_cond: bool = False):
    """Rows of A in path order: (rowptr int64 (n+1,), j int32, chord mm float64, margin (n,)).

    A row lists the visits of the MLP polyline (maximal runs inside one voxel)
    in hull voxels, in the order the path meets them; ``margin`` is the
    smallest distance (mm) from a crossing, a turning vertex or the sample-count
    boundary to a voxel face -- rows below 1e-4 mm are near-face cases.
    With ``with_cond`` a fifth array gives, per row, the largest ratio of
    segment length to its extent across a crossed face (how much a sideways
    position error moves a crossing along the path; 1 for a head-on crossing),
    over the walk's crossings and the tracker lines' crossings into their first
    hull voxels.
    """
    keep, arr, n = _hist_arrays(hist)
    rowptr = np.zeros(n + 1, dtype=np.int64)
    margin = np.zeros(n)
    cond = np.ones(n)
    lib = _L()
    lib.o_rows(geo._cp(), geo._mp(), n, arr, _ptr(rowptr), None, None, _ptr(margin), _ptr(cond))
    np.cumsum(rowptr, out=rowptr)
    nnz = int(rowptr[-1])
    j = np.zeros(max(nnz, 1), dtype=np.int32)
    ln = np.zeros(max(nnz, 1))
    if lib.o_rows(geo._cp(), geo._mp(), n, arr, _ptr(rowptr), _ptr(j), _ptr(ln), _ptr(margin),
                  _ptr(cond)) != 0:
        raise RuntimeError("oracle row count changed between passes")
    del keep
    if with_cond:
        return rowptr, j[:nnz], ln[:nnz], margin, cond
    return rowptr, j[:nnz], ln[:nnz], margin


def walk(geo: Geometry, pts, cap: int = 100000):
    """Row of one caller-given polyline (lab mm, shape (np, 3)): (j, chord, margin)."""
    p = np.ascontiguousarray(pts, dtype=np.float64).reshape(-1, 3)
    j = np.zeros(cap, dtype=np.int32)
    ln = np.zeros(cap)
    m = np.full(1, np.inf)
    k = _L().o_walk(geo._cp(), geo._mp(), p.shape[0], _ptr(p), _ptr(j), _ptr(ln), cap, _ptr(m))
    if k > cap:
        raise ValueError("row longer than cap")
    return j[:k].copy(), ln[:k].copy(), float(m[0])


def csr(rowptr, j, ln, n_vox: int):
    """A as a scipy CSR matrix (m x n_vox) with repeated (i, j) entries summed."""
    import scipy.sparse as sp
    m = rowptr.size - 1
    # copies: scipy would otherwise share the caller's arrays, and summing
    # duplicates sorts each row in place
    A = sp.csr_matrix((np.array(ln, dtype=np.float64), np.array(j, dtype=np.int64),
                       np.array(rowptr, dtype=np.int64)), shape=(m, n_vox))
    A.sum_duplicates()
    A.eliminate_zeros()
    return A


def drop(A, b, iters: int, lam: float, block: int, x0) -> np.ndarray:
    """DROP (Sec. IV-B): ``iters`` passes over blocks of ``block`` consecutive rows."""
    A = A.tocsr(copy=True)
    A.sum_duplicates()
    A.eliminate_zeros()
    rowptr = np.ascontiguousarray(A.indptr, dtype=np.int64)
    idx = np.ascontiguousarray(A.indices, dtype=np.int32)
    val = np.ascontiguousarray(A.data, dtype=np.float64)
    bb = np.ascontiguousarray(b, dtype=np.float64)
    x = np.array(x0, dtype=np.float64, copy=True)
    if bb.size != A.shape[0] or x.size != A.shape[1]:
        raise ValueError("shape mismatch")
    rc = _L().o_drop(A.shape[1], A.shape[0], _ptr(rowptr), _ptr(idx), _ptr(val), _ptr(bb),
                     int(iters), float(lam), int(block), _ptr(x))
    if rc != 0:
        raise ValueError("o_drop failed (%d)" % rc)
    return x


def forward(A, x) -> np.ndarray:
    """y = A x in FP64."""
    return A @ np.asarray(x, dtype=np.float64)


def adjoint(A, y) -> np.ndarray:
    """g = A^T y in FP64."""
    return A.T @ np.asarray(y, dtype=np.float64)


def tv(x, shape, eps: float = 1e-6):
    """Isotropic TV(x) = sum_v sqrt(|D+ x|_v^2 + eps^2) and its gradient.

    D+ is the forward difference along x, y and z with a zero difference at
    the last index of each axis (Neumann boundary).  ``shape`` = (nx, ny, nz);
    x is flat in j order.
    """
    nx, ny, nz = shape
    v = np.asarray(x, dtype=np.float64).reshape(nz, ny, nx)
    gx = np.zeros_like(v)
    gy = np.zeros_like(v)
    gz = np.zeros_like(v)
    gx[:, :, :-1] = v[:, :, 1:] - v[:, :, :-1]
    gy[:, :-1, :] = v[:, 1:, :] - v[:, :-1, :]
    gz[:-1, :, :] = v[1:, :, :] - v[:-1, :, :]
    mag = np.sqrt(gx * gx + gy * gy + gz * gz + eps * eps)
    val = float(mag.sum())
    px, py, pz = gx / mag, gy / mag, gz / mag
    grad = -(px + py + pz)
    grad[:, :, 1:] += px[:, :, :-1]
    grad[:, 1:, :] += py[:, :-1, :]
    grad[1:, :, :] += pz[:-1, :, :]
    return val, grad.reshape(-1)
