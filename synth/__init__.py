"""Seeded synthetic proton-CT scans (phantoms, hull masks and proton histories).

This module is the one input source that both the CUDA path and the FP64
oracle read.  It holds none of the reconstruction arithmetic: it does not
compute a most likely path, a voxel walk, a scattering matrix or a DROP
update.  It simulates the measurement instead -- a proton random walk through
a voxelised analytic phantom with multiple-scattering kicks and a residual
range model, the WEPL taken as the midpoint-rule integral of the true RSP
along the simulated path -- to stand in for the paper's Geant4-simulated and
experimental CTP404 scans (Sec. IV-A), which are not available.  Shapes,
sizes, angle steps and proton counts follow the workloads the reconstruction
is quoted on (20 slices of 0.25 cm, 4-degree steps, 1e5 ... 2.61e8 protons).

Everything runs in torch on the device passed in ("cpu" for tests, "cuda" for
full-size benchmarks); the same seed gives the same scan on a given device.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np
import torch

HIST_FIELDS = ("in_x", "in_y", "in_z", "out_x", "out_y", "out_z",
               "theta_in", "psi_in", "theta_out", "psi_out", "phi", "wepl")

SEED_BASE = 180201070

# measurement model constants (simulation only)
_MP = 938.272          # proton mass, MeV
_HL = 13.6             # Highland constant, MeV
_X0 = 36.08            # radiation length of water, cm
_BK_ALPHA = 0.0022     # Bragg-Kleeman range-energy rule R = alpha E^p (cm, MeV), water
_BK_P = 1.77
_E_FLOOR = 30.0        # MeV; protons that would range out keep this energy


@dataclass
class ScanConfig:
    name: str
    shape: tuple          # (nx, ny, nz)
    voxel: float          # mm, cubic voxels
    phantom: str          # "tiny" | "head" | "torso" | "ellipsoids"
    n_protons: int
    n_angles: int
    iters: int
    lam: float
    block: int
    energy: float = 200.0
    angle_sigma: float = 5e-3
    wepl_noise: float = 0.01
    seed_offset: int = 0
    extra: dict = field(default_factory=dict)

    @property
    def n_vox(self):
        return self.shape[0] * self.shape[1] * self.shape[2]

    @property
    def origin(self):
        return tuple(-0.5 * n * self.voxel for n in self.shape)

    @property
    def seed(self):
        return SEED_BASE + self.seed_offset


# The five workloads: a tiny plain reconstruction, a head-sized stored-row
# solve, a torso-sized fused solve, a differentiable-projector scan and a large
# torso; lambda where the workload does not fix one is 0.5 (a reading).
CONFIGS = {
    "tiny": ScanConfig("tiny", (64, 64, 8), 1.0, "tiny", 100_000, 90, 6, 1e-4, 3200, seed_offset=0),
    "head": ScanConfig("head", (200, 200, 32), 1.0, "head", 10_000_000, 90, 12, 0.5, 3200,
                       seed_offset=1),
    "torso": ScanConfig("torso", (280, 280, 96), 1.0, "torso", 116_000_000, 180, 6, 0.5, 320_000,
                        seed_offset=2),
    "diff": ScanConfig("diff", (128, 128, 32), 1.0, "ellipsoids", 4_000_000, 90, 50, 0.0, 0,
                       seed_offset=3),
    "large": ScanConfig("large", (320, 320, 128), 1.0, "torso", 261_000_000, 180, 6, 0.5, 320_000,
                        seed_offset=4),
}


def validation_scans(count: int = 16, n_min: float = 1e5, n_max: float = 2e6, seed_offset: int = 10):
    """Small scans of uneven size for batched solves: proton counts log-uniform
    in [n_min, n_max], grids between 64x64x8 and 128x128x32 (1 mm), seeded
    ellipsoid phantoms, 90 angles, 6 DROP iterations, block 3200."""
    g = torch.Generator().manual_seed(SEED_BASE + seed_offset)
    out = []
    for k in range(count):
        u = torch.rand(3, generator=g, dtype=torch.float64)
        n = int(round(math.exp(math.log(n_min) + (math.log(n_max) - math.log(n_min)) * u[0].item())))
        nx = (64, 96, 128)[int(u[1].item() * 3) % 3]
        nz = (8, 16, 32)[int(u[2].item() * 3) % 3]
        out.append(ScanConfig("scan%02d" % k, (nx, nx, nz), 1.0, "ellipsoids", n, 90, 6, 0.5, 3200,
                              seed_offset=seed_offset + 1 + k))
    return out


def scaled(cfg: ScanConfig, n_protons: int, name: str | None = None, **kw) -> ScanConfig:
    """A copy of ``cfg`` with another proton count (same phantom, beam and seed)."""
    d = dict(cfg.__dict__)
    d.update(kw)
    d["n_protons"] = int(n_protons)
    d["name"] = name or "%s@%d" % (cfg.name, n_protons)
    d["extra"] = dict(cfg.extra)
    return ScanConfig(**d)


# --------------------------------------------------------------------------
# Phantoms
# --------------------------------------------------------------------------

def _centres(shape, voxel):
    nx, ny, nz = shape
    xs = (torch.arange(nx, dtype=torch.float64) + 0.5 - nx / 2) * voxel
    ys = (torch.arange(ny, dtype=torch.float64) + 0.5 - ny / 2) * voxel
    zs = (torch.arange(nz, dtype=torch.float64) + 0.5 - nz / 2) * voxel
    z, y, x = torch.meshgrid(zs, ys, xs, indexing="ij")
    return x, y, z


def _ellipsoid(x, y, z, c, a, rot=0.0):
    cr, sr = math.cos(rot), math.sin(rot)
    dx, dy, dz = x - c[0], y - c[1], z - c[2]
    px, py = cr * dx + sr * dy, -sr * dx + cr * dy
    return (px / a[0]) ** 2 + (py / a[1]) ** 2 + (dz / a[2]) ** 2 <= 1.0


def _ellcyl(x, y, c, a):
    return ((x - c[0]) / a[0]) ** 2 + ((y - c[1]) / a[1]) ** 2 <= 1.0


def phantom(cfg: ScanConfig):
    """(rsp float32 (n_vox,), hull uint8 (n_vox,)) in j = ix + nx (iy + ny iz) order.

    The voxel value is the RSP at the voxel centre; the hull is the body shape.
    """
    x, y, z = _centres(cfg.shape, cfg.voxel)
    g = torch.Generator().manual_seed(cfg.seed)
    rsp = torch.zeros_like(x)
    kind = cfg.phantom
    if kind == "tiny":
        body = _ellcyl(x, y, (0, 0), (28.0, 28.0))
        rsp[body] = 1.0
        for k, val in enumerate((0.3, 1.1, 1.6)):
            a = 2 * math.pi * k / 3
            m = _ellipsoid(x, y, z, (14 * math.cos(a), 14 * math.sin(a), 0.0), (6.0, 6.0, 3.0))
            rsp[m & body] = val
    elif kind == "head":
        body = _ellipsoid(x, y, z, (0, 0, 0), (90.0, 75.0, 15.0))
        rsp[body] = 1.04
        vals = (0.25, 0.95, 1.04, 1.6)
        for _ in range(11):
            u = torch.rand(8, generator=g, dtype=torch.float64)
            c = ((u[0] - 0.5) * 110, (u[1] - 0.5) * 90, (u[2] - 0.5) * 14)
            a = (6 + 18 * u[3].item(), 6 + 15 * u[4].item(), 3 + 6 * u[5].item())
            m = _ellipsoid(x, y, z, c, a, rot=math.pi * u[6].item())
            rsp[m & body] = vals[int(u[7].item() * 4) % 4]
    elif kind == "torso":
        body = _ellcyl(x, y, (0, 0), (130.0, 100.0))
        rsp[body] = 1.0
        hz = 0.5 * cfg.shape[2] * cfg.voxel
        for sx in (-1, 1):
            m = _ellipsoid(x, y, z, (sx * 60.0, 5.0, 0.0), (45.0, 60.0, hz * 1.2))
            rsp[m & body] = 0.3
        spine = _ellcyl(x, y, (0.0, -70.0), (14.0, 14.0))
        rsp[spine & body] = 1.6
        for _ in range(6):
            u = torch.rand(6, generator=g, dtype=torch.float64)
            c = ((u[0] - 0.5) * 200, (u[1] - 0.5) * 150, (u[2] - 0.5) * hz)
            a = (5 + 12 * u[3].item(), 5 + 12 * u[4].item(), 5 + 20 * u[5].item())
            m = _ellipsoid(x, y, z, c, a)
            rsp[m & body] = 1.6
    elif kind == "ellipsoids":
        nx = cfg.shape[0]
        r = 0.44 * nx * cfg.voxel
        hz = 0.5 * cfg.shape[2] * cfg.voxel
        body = _ellcyl(x, y, (0, 0), (r, r))
        rsp[body] = 1.0
        vals = (0.25, 0.95, 1.04, 1.6)
        for _ in range(8):
            u = torch.rand(8, generator=g, dtype=torch.float64)
            c = ((u[0] - 0.5) * r, (u[1] - 0.5) * r, (u[2] - 0.5) * hz)
            a = (3 + 0.2 * r * u[3].item(), 3 + 0.2 * r * u[4].item(), 2 + 0.4 * hz * u[5].item())
            m = _ellipsoid(x, y, z, c, a, rot=math.pi * u[6].item())
            rsp[m & body] = vals[int(u[7].item() * 4) % 4]
    else:
        raise ValueError("unknown phantom %r" % kind)
    hull = body.to(torch.uint8)
    return rsp.to(torch.float32).reshape(-1), hull.reshape(-1)


# --------------------------------------------------------------------------
# Proton histories
# --------------------------------------------------------------------------

def tracker_half_span(cfg: ScanConfig) -> float:
    """U: trackers sit at depth -U and +U, U = half the x-y grid diagonal + 10 mm."""
    nx, ny, _ = cfg.shape
    return 0.5 * math.hypot(nx * cfg.voxel, ny * cfg.voxel) + 10.0


def _lookup(rsp_grid, cfg, x, y, z):
    nx, ny, nz = cfg.shape
    o = cfg.origin
    ix = torch.floor((x - o[0]) / cfg.voxel).to(torch.int64)
    iy = torch.floor((y - o[1]) / cfg.voxel).to(torch.int64)
    iz = torch.floor((z - o[2]) / cfg.voxel).to(torch.int64)
    inside = (ix >= 0) & (ix < nx) & (iy >= 0) & (iy < ny) & (iz >= 0) & (iz < nz)
    j = (ix.clamp(0, nx - 1) + nx * (iy.clamp(0, ny - 1) + ny * iz.clamp(0, nz - 1)))
    return torch.where(inside, rsp_grid[j], torch.zeros((), dtype=rsp_grid.dtype, device=x.device))


def _simulate(cfg, rsp_grid, phi, t, v, th, ps, gen, step_mm):
    """Random walk from depth -U to +U; returns exit (t, v, th, ps) and WEPL (mm)."""
    dev = t.device
    U = tracker_half_span(cfg)
    c, s = torch.cos(phi), torch.sin(phi)
    wepl = torch.zeros_like(t)
    r0 = _BK_ALPHA * cfg.energy ** _BK_P
    log_ref = 1.0 + 0.038 * math.log(max(0.15 * cfg.shape[0] * cfg.voxel, 1.0) / _X0)
    n_steps = int(math.ceil(2 * U / step_mm))
    h = 2 * U / n_steps
    u = -U
    for _ in range(n_steps):
        tt, tp = torch.tan(th), torch.tan(ps)
        um = u + 0.5 * h
        tm, vm = t + 0.5 * h * tt, v + 0.5 * h * tp
        rho = _lookup(rsp_grid, cfg, um * c - tm * s, um * s + tm * c, vm)
        seg = h * torch.sqrt(1.0 + tt * tt + tp * tp)
        wet_cm = 0.1 * seg * rho
        res = (r0 - 0.1 * wepl).clamp_min(_BK_ALPHA * _E_FLOOR ** _BK_P)
        e = (res / _BK_ALPHA) ** (1.0 / _BK_P)
        pv = (e * e + 2 * e * _MP) / (e + _MP)          # beta c p, MeV
        sig = (_HL / pv) * torch.sqrt(wet_cm / _X0) * log_ref
        t = t + h * tt
        v = v + h * tp
        th = th + sig * torch.randn(t.shape, generator=gen, device=dev, dtype=t.dtype)
        ps = ps + sig * torch.randn(t.shape, generator=gen, device=dev, dtype=t.dtype)
        wepl = wepl + seg * rho
        u += h
    return t, v, th, ps, wepl


def histories(cfg: ScanConfig, device="cpu", n: int | None = None, chunk: int = 1 << 22,
              step_mm: float = 1.0, rsp=None, outlier_frac: float = 0.0):
    """Proton histories as a dict of float32 tensors on ``device``.

    Proton i takes gantry angle index i mod n_angles (angles k * 360/n_angles
    degrees), then the storage order is shuffled with the scan's seed.  Entry
    tracker points are uniform over the detector face (t over the x extent, v
    over the z extent) at depth -U, entry angles N(0, angle_sigma); exit points
    and angles come from the random walk at depth +U; WEPL gets Gaussian noise
    of ``wepl_noise`` times its value.

    ``outlier_frac`` > 0 corrupts that fraction of the protons (drawn from a
    generator of its own, so every other proton is unchanged) the way
    nuclear interactions and large-angle scatters corrupt measured data: half
    of them get a WEPL 15-60 % too large, the other half an exit angle off by
    80-250 mrad in theta or psi.  ``outlier_mask`` (below) returns which.
    """
    n = cfg.n_protons if n is None else int(n)
    dev = torch.device(device)
    if rsp is None:
        rsp, _ = phantom(cfg)
    rsp_grid = rsp.to(dev, torch.float32)
    gen = torch.Generator(device=dev).manual_seed(cfg.seed)
    perm = torch.randperm(n, generator=gen, device=dev)
    U = tracker_half_span(cfg)
    half_t = 0.5 * cfg.shape[0] * cfg.voxel
    half_v = 0.5 * cfg.shape[2] * cfg.voxel
    out = {k: torch.empty(n, dtype=torch.float32, device=dev) for k in HIST_FIELDS}
    for a in range(0, n, chunk):
        b = min(n, a + chunk)
        m = b - a
        idx = perm[a:b]
        phi = (idx % cfg.n_angles).to(torch.float32) * (2 * math.pi / cfg.n_angles)
        t = (torch.rand(m, generator=gen, device=dev) * 2 - 1) * half_t
        v = (torch.rand(m, generator=gen, device=dev) * 2 - 1) * half_v
        th = torch.randn(m, generator=gen, device=dev) * cfg.angle_sigma
        ps = torch.randn(m, generator=gen, device=dev) * cfg.angle_sigma
        t2, v2, th2, ps2, wepl = _simulate(cfg, rsp_grid, phi, t, v, th, ps, gen, step_mm)
        wepl = wepl + cfg.wepl_noise * wepl * torch.randn(m, generator=gen, device=dev)
        c, s = torch.cos(phi), torch.sin(phi)
        out["in_x"][a:b] = -U * c - t * s
        out["in_y"][a:b] = -U * s + t * c
        out["in_z"][a:b] = v
        out["out_x"][a:b] = U * c - t2 * s
        out["out_y"][a:b] = U * s + t2 * c
        out["out_z"][a:b] = v2
        out["theta_in"][a:b] = th
        out["psi_in"][a:b] = ps
        out["theta_out"][a:b] = th2
        out["psi_out"][a:b] = ps2
        out["phi"][a:b] = phi
        out["wepl"][a:b] = wepl
    if outlier_frac > 0.0:
        bad, kind, mag, sgn = _outliers(cfg, n, dev, outlier_frac)
        w = out["wepl"]
        out["wepl"] = torch.where(bad & (kind == 0), w * (1.15 + 0.45 * mag), w)
        kick = sgn * (0.08 + 0.17 * mag)
        out["theta_out"] = torch.where(bad & (kind == 1), out["theta_out"] + kick, out["theta_out"])
        out["psi_out"] = torch.where(bad & (kind == 2), out["psi_out"] + kick, out["psi_out"])
    return out


def _outliers(cfg, n, dev, frac):
    g = torch.Generator(device=dev).manual_seed(cfg.seed + 7_654_321)
    bad = torch.rand(n, generator=g, device=dev) < frac
    kind = (torch.rand(n, generator=g, device=dev) * 4).to(torch.int64).clamp_max(3)
    kind = torch.where(kind >= 2, kind - 1, torch.zeros_like(kind))   # 0: WEPL (half), 1: theta, 2: psi
    mag = torch.rand(n, generator=g, device=dev)
    sgn = torch.where(torch.rand(n, generator=g, device=dev) < 0.5, -1.0, 1.0)
    return bad, kind, mag, sgn


def outlier_mask(cfg: ScanConfig, n: int | None = None, frac: float = 0.02, device="cpu"):
    """Which protons ``histories(..., outlier_frac=frac)`` corrupted (bool tensor)."""
    n = cfg.n_protons if n is None else int(n)
    return _outliers(cfg, n, torch.device(device), frac)[0]


def clean_bins(cfg: ScanConfig) -> dict:
    """Bins of the data-cleaning step for a scan: one per gantry angle, t over the
    detector width and v over its height, 1 x 2.5 mm (the paper's 0.25 cm
    slices) for the large scans; for small ones v, then t, bins are doubled
    until a bin holds some 30 protons."""
    nx, _, nz = cfg.shape
    half_t = 0.5 * nx * cfg.voxel
    half_v = 0.5 * nz * cfg.voxel
    per = cfg.n_protons / cfg.n_angles
    dt, dv = cfg.voxel, 2.5 * cfg.voxel

    def fill(dt, dv):
        return per / (math.ceil(2 * half_t / dt) * math.ceil(2 * half_v / dv))

    while fill(dt, dv) < 30 and dv < 2 * half_v:      # taller bins first: WEPL varies least along v
        dv *= 2
    while fill(dt, dv) < 30 and dt < half_t:
        dt *= 2
    n_t = int(math.ceil(2 * half_t / dt))
    n_v = max(int(math.ceil(2 * half_v / dv)), 1)
    return {"n_angle": cfg.n_angles, "angle_step": 2 * math.pi / cfg.n_angles, "n_t": n_t,
            "t_min": -0.5 * n_t * dt, "dt": dt, "n_v": n_v, "v_min": -0.5 * n_v * dv, "dv": dv,
            "k_sigma": 3.0}


def to_numpy(hist):
    """float32 numpy copies of a history dict (host memory)."""
    return {k: (v.detach().cpu().numpy() if torch.is_tensor(v) else np.asarray(v, dtype=np.float32))
            for k, v in hist.items()}


def subset(hist, start, stop):
    return {k: v[start:stop] for k, v in hist.items()}


def fbp_bins(cfg: ScanConfig) -> dict:
    """Sinogram bins of the FBP initial iterate for a scan: one per gantry angle,
    t bins of one voxel over the detector width, v bins of one voxel aligned
    with the grid's slices."""
    nx, _, nz = cfg.shape
    return {"n_angle": cfg.n_angles, "angle_step": 2 * math.pi / cfg.n_angles, "n_t": nx,
            "t_min": -0.5 * nx * cfg.voxel, "dt": cfg.voxel, "n_v": nz, "v_min": cfg.origin[2],
            "dv": cfg.voxel}
