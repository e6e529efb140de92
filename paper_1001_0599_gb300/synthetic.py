"""Seeded synthetic inputs: workloads, ellipsoid phantoms, exact sinograms, noise.

This module generates inputs only. It holds none of the reconstruction
method's arithmetic (no discrete projector, no TV, no solver): the sinogram it
produces is the exact line integral of an analytic ellipsoid phantom, i.e. a
simulated scanner, and both the CUDA path and the FP64 oracle consume it.

The paper's own data (an NCAT thorax phantom, a CatPhan 600, a Rando head
phantom and a patient scan; Sec. III) are not available, so seeded ellipsoid
phantoms with the shapes and attenuation ranges of those workloads stand in
for them. Geometry follows the circular cone-beam set-up of Fig. 1 / Eq. (A2):
source on a circle of radius ``sad`` in the z = 0 plane, flat detector at
distance ``sdd`` from the source, u axis along -y at angle 0, v along +z.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Sequence

import numpy as np


# ----------------------------------------------------------------------------
# Workload descriptions
# ----------------------------------------------------------------------------

@dataclasses.dataclass
class Workload:
    """Sizes and physics of one synthetic reconstruction problem."""

    name: str
    nx: int
    ny: int
    nz: int
    dx: float
    dy: float
    dz: float
    nu: int
    nv: int
    du: float
    dv: float
    n_views: int
    sad: float = 1000.0
    sdd: float = 1500.0
    arc_deg: float = 360.0
    photons: float = 1e5
    phantom: str = "ellipsoids"      # "ellipsoids" | "head_neck"
    phantom_seed: int = 1
    noise_seed: int = 2
    lam: float = 0.05
    iters: Sequence[int] = (10,)      # FBS iterations per multigrid level, coarse -> fine
    step_ratio: float = 0.5

    @property
    def angles(self) -> np.ndarray:
        # evenly spaced over the arc; for a full circle the end point is excluded
        k = np.arange(self.n_views, dtype=np.float64)
        return np.deg2rad(self.arc_deg) * k / self.n_views

    @property
    def n_levels(self) -> int:
        return len(self.iters)

    def scaled(self, factor: int) -> "Workload":
        """Same physics on a grid coarser by ``factor`` per axis (for quick tests)."""
        return dataclasses.replace(
            self, nx=self.nx // factor, ny=self.ny // factor, nz=self.nz // factor,
            dx=self.dx * factor, dy=self.dy * factor, dz=self.dz * factor)


def workload(name: str) -> Workload:
    """The five synthetic workloads (sizes of the paper's experiments, Sec. III).

    small      -- 64^3 at 2 mm, 128x96 detector at 0.8 mm, 40 views, 1e5 photons,
                  10 FBS iterations, lambda 0.05, no multigrid.
    paper      -- 256x256x128 at 1 mm, 512x384 detector at 0.78 mm, 40 views,
                  head-and-neck-like phantom, 5e4 photons, 3-level multigrid
                  (64 -> 128 -> 256 in-plane), 100 FBS iterations (40/30/30).
    lowdose    -- 256^3 at 1 mm, 512x384 detector, 360 views, 1e4 photons.
    cube40     -- 256^3 at 1 mm, 512x384 detector, 40 views, 5e4 photons, 3-level
                  multigrid (40/30/30): the paper-scale schedule on a cubic volume.
    autograd   -- 128^3 at 2 mm, 256x192 detector at 1.56 mm, 60 views.
    """
    if name == "small":
        return Workload("small", 64, 64, 64, 2.0, 2.0, 2.0, 128, 96, 0.8, 0.8, 40,
                        photons=1e5, phantom="ellipsoids", phantom_seed=1, noise_seed=2,
                        lam=0.05, iters=(10,))
    if name == "paper":
        return Workload("paper", 256, 256, 128, 1.0, 1.0, 1.0, 512, 384, 0.78, 0.78, 40,
                        photons=5e4, phantom="head_neck", phantom_seed=3, noise_seed=4,
                        lam=0.05, iters=(40, 30, 30))
    if name == "lowdose":
        return Workload("lowdose", 256, 256, 256, 1.0, 1.0, 1.0, 512, 384, 0.78, 0.78, 360,
                        photons=1e4, phantom="head_neck", phantom_seed=5, noise_seed=6,
                        lam=0.05, iters=(40, 30, 30))
    if name == "cube40":
        return Workload("cube40", 256, 256, 256, 1.0, 1.0, 1.0, 512, 384, 0.78, 0.78, 40,
                        photons=5e4, phantom="head_neck", phantom_seed=5, noise_seed=6,
                        lam=0.05, iters=(40, 30, 30))
    if name == "autograd":
        return Workload("autograd", 128, 128, 128, 2.0, 2.0, 2.0, 256, 192, 1.56, 1.56, 60,
                        photons=5e4, phantom="head_neck", phantom_seed=7, noise_seed=8,
                        lam=0.05, iters=(10,))
    raise KeyError(name)


# ----------------------------------------------------------------------------
# Phantoms
# ----------------------------------------------------------------------------

@dataclasses.dataclass
class Ellipsoid:
    centre: np.ndarray     # (3,) mm
    axes: np.ndarray       # (3,) semi-axes, mm
    phi: float             # rotation about z, radians
    value: float           # additive attenuation contrast, 1/mm


def _rot_z(phi: float) -> np.ndarray:
    c, s = math.cos(phi), math.sin(phi)
    return np.array([[c, -s, 0.0], [s, c, 0.0], [0.0, 0.0, 1.0]])


def _place(rng: np.random.Generator, body: Ellipsoid, placed: List[Ellipsoid],
           n: int, axes_lo: float, axes_hi: float, values, tries: int = 20000) -> None:
    """Rejection-sample ``n`` ellipsoids inside ``body`` whose bounding spheres
    neither overlap each other nor leave the body."""
    got = 0
    for _ in range(tries):
        if got == n:
            return
        ax = rng.uniform(axes_lo, axes_hi, size=3)
        ax[2] = min(ax[2], 0.8 * body.axes[2])
        r = float(ax.max())
        # candidate centre inside the body shrunk by r (sufficient for containment)
        shrunk = body.axes - r
        if np.any(shrunk <= 0):
            continue
        p = rng.uniform(-1.0, 1.0, size=3)
        if float(np.sum(p * p)) > 1.0:
            continue
        c = body.centre + p * shrunk
        if any(np.linalg.norm(c - e.centre) < r + float(e.axes.max()) + 1.0 for e in placed):
            continue
        v = float(values(rng)) if callable(values) else float(values)
        placed.append(Ellipsoid(c, ax, float(rng.uniform(0, math.pi)), v))
        got += 1
    raise RuntimeError("could not place ellipsoids")


def make_phantom(wl: Workload) -> List[Ellipsoid]:
    """Seeded ellipsoid phantom for a workload; contrasts are additive.

    The first ellipsoid is the body; every other one lies inside it and carries
    (its attenuation - body attenuation) so that sums of chords give the
    piecewise-constant attenuation map.
    """
    rng = np.random.default_rng(wl.phantom_seed)
    if wl.phantom == "ellipsoids":
        # body kept inside the detector's field of view (radius ~34 mm, |z| ~25 mm
        # at the isocentre for the small workload)
        fov_r = wl.sad * math.sin(math.atan(0.5 * wl.nu * wl.du / wl.sdd))
        fov_z = 0.5 * wl.nv * wl.dv * (wl.sad - fov_r) / wl.sdd
        bx = min(30.0, 0.88 * fov_r, 0.45 * wl.nx * wl.dx)
        body = Ellipsoid(np.zeros(3), np.array([bx, 0.87 * bx, min(20.0, 0.8 * fov_z, 0.45 * wl.nz * wl.dz)]),
                         0.0, 0.02)
        inner: List[Ellipsoid] = []
        lo, hi = 0.08 * bx, 0.22 * bx
        _place(rng, body, inner, 10, lo, hi, lambda r: r.uniform(0.01, 0.03))
        for e in inner:
            e.value -= body.value
        return [body] + inner
    if wl.phantom == "head_neck":
        fov_r = wl.sad * math.sin(math.atan(0.5 * wl.nu * wl.du / wl.sdd))
        half = np.array([wl.nx * wl.dx, wl.ny * wl.dy, wl.nz * wl.dz]) * 0.5
        bx = min(0.62 * fov_r, 0.62 * half[0])
        body = Ellipsoid(np.zeros(3), np.array([bx, 1.2 * bx, 0.9 * half[2]]), 0.0, 0.019)
        inner = []
        _place(rng, body, inner, 6, 0.06 * bx, 0.2 * bx, 0.04)     # bone
        _place(rng, body, inner, 4, 0.06 * bx, 0.16 * bx, 0.0)     # air cavities
        for e in inner:
            e.value -= body.value
        return [body] + inner
    raise KeyError(wl.phantom)


def _inside(e: Ellipsoid, x: np.ndarray, y: np.ndarray, z: np.ndarray) -> np.ndarray:
    c, s = math.cos(e.phi), math.sin(e.phi)
    px, py, pz = x - e.centre[0], y - e.centre[1], z - e.centre[2]
    qx = c * px + s * py
    qy = -s * px + c * py
    return (qx / e.axes[0]) ** 2 + (qy / e.axes[1]) ** 2 + (pz / e.axes[2]) ** 2 <= 1.0


def voxelise(ells: Sequence[Ellipsoid], nx: int, ny: int, nz: int,
             dx: float, dy: float, dz: float, ss: int = 4) -> np.ndarray:
    """Ground-truth volume [nx][ny][nz] (z fastest): mean of ``ss``^3 sub-samples
    of the piecewise-constant phantom in each voxel. Voxels far from every
    surface are filled from their centre; only boundary voxels are sub-sampled."""
    xs = (np.arange(nx) - 0.5 * (nx - 1)) * dx
    ys = (np.arange(ny) - 0.5 * (ny - 1)) * dy
    zs = (np.arange(nz) - 0.5 * (nz - 1)) * dz
    vol = np.zeros((nx, ny, nz), dtype=np.float64)
    offs = (np.arange(ss) + 0.5) / ss - 0.5
    half_diag = 0.5 * math.sqrt(dx * dx + dy * dy + dz * dz)
    for e in ells:
        r = float(e.axes.max()) + half_diag
        ia = np.nonzero(np.abs(xs - e.centre[0]) <= r)[0]
        ib = np.nonzero(np.abs(ys - e.centre[1]) <= r)[0]
        ic = np.nonzero(np.abs(zs - e.centre[2]) <= r)[0]
        if len(ia) == 0 or len(ib) == 0 or len(ic) == 0:
            continue
        X, Y, Z = np.meshgrid(xs[ia], ys[ib], zs[ic], indexing="ij")
        # scaled radial coordinate at the voxel centre decides interior/exterior
        c, s = math.cos(e.phi), math.sin(e.phi)
        px, py, pz = X - e.centre[0], Y - e.centre[1], Z - e.centre[2]
        qx, qy = c * px + s * py, -s * px + c * py
        rho = np.sqrt((qx / e.axes[0]) ** 2 + (qy / e.axes[1]) ** 2 + (pz / e.axes[2]) ** 2)
        margin = half_diag / float(e.axes.min())
        occ = (rho <= 1.0).astype(np.float64)
        edge = np.abs(rho - 1.0) <= margin * 1.05 + 1e-12
        if np.any(edge):
            ex, ey, ez = X[edge], Y[edge], Z[edge]
            acc = np.zeros(ex.shape[0])
            for ox in offs:
                for oy in offs:
                    for oz in offs:
                        acc += _inside(e, ex + ox * dx, ey + oy * dy, ez + oz * dz)
            occ[edge] = acc / ss ** 3
        vol[np.ix_(ia, ib, ic)] += e.value * occ
    return vol


# ----------------------------------------------------------------------------
# Exact line integrals (simulated scanner) and noise
# ----------------------------------------------------------------------------

def ray_endpoints(wl: Workload):
    """Source positions (n_views, 3) and detector pixel centres
    (n_views, nv, nu, 3) for the circular orbit (Fig. 1, Eq. A2 at angle 0)."""
    th = wl.angles
    c, s = np.cos(th), np.sin(th)
    src = np.stack([-wl.sad * c, -wl.sad * s, np.zeros_like(c)], axis=1)
    u = (np.arange(wl.nu) - 0.5 * (wl.nu - 1)) * wl.du
    v = (np.arange(wl.nv) - 0.5 * (wl.nv - 1)) * wl.dv
    det = np.empty((wl.n_views, wl.nv, wl.nu, 3))
    off = wl.sdd - wl.sad
    det[..., 0] = (off * c)[:, None, None] + u[None, None, :] * s[:, None, None]
    det[..., 1] = (off * s)[:, None, None] - u[None, None, :] * c[:, None, None]
    det[..., 2] = v[None, :, None]
    return src, det


def exact_sinogram(ells: Sequence[Ellipsoid], wl: Workload) -> np.ndarray:
    """Line integrals of the analytic phantom along every source-to-pixel ray,
    [n_views][nv][nu] (u fastest), FP64."""
    src, det = ray_endpoints(wl)
    out = np.zeros((wl.n_views, wl.nv, wl.nu))
    for k in range(wl.n_views):
        S = src[k]
        d = det[k] - S
        d = d / np.linalg.norm(d, axis=-1, keepdims=True)
        for e in ells:
            R = _rot_z(-e.phi)
            s0 = (R @ (S - e.centre)) / e.axes
            dd = (d @ R.T) / e.axes
            A = np.sum(dd * dd, axis=-1)
            B = dd @ s0
            C = float(s0 @ s0) - 1.0
            disc = B * B - A * C
            chord = np.where(disc > 0, 2.0 * np.sqrt(np.maximum(disc, 0.0)) / A, 0.0)
            out[k] += e.value * chord
    return out


def poisson_log_sinogram(p: np.ndarray, photons: float, seed: int) -> np.ndarray:
    """Noisy measured line integrals y = ln(N0 / max(N, 1)), N ~ Poisson(N0 e^-p)."""
    rng = np.random.default_rng(seed)
    counts = rng.poisson(photons * np.exp(-p))
    return np.log(photons / np.maximum(counts, 1))


def make_problem(wl: Workload, noise: bool = True):
    """(ground-truth volume, measured sinogram) for a workload, both FP64."""
    ells = make_phantom(wl)
    truth = voxelise(ells, wl.nx, wl.ny, wl.nz, wl.dx, wl.dy, wl.dz)
    p = exact_sinogram(ells, wl)
    y = poisson_log_sinogram(p, wl.photons, wl.noise_seed) if noise else p
    return truth, y


def random_volume(shape, seed: int, low: float = 0.0, high: float = 1.0) -> np.ndarray:
    return np.random.default_rng(seed).uniform(low, high, size=shape)
