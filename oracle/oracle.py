"""Python front end of the FP64 CPU oracle (TEST INFRASTRUCTURE ONLY).

Only the tests, the smoke check and the CPU-baseline leg of the benchmark may
import this module. It wraps ``cbct_oracle.c`` (plain C, FP64, OpenMP) through
ctypes and adds the multigrid driver of Sec. II.C.3, written out plainly.
Nothing here is shared with, or imported by, the CUDA library.
"""
from __future__ import annotations

import ctypes
import dataclasses
import os
import subprocess
from typing import List, Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "cbct_oracle.c")
_HDR = os.path.join(_HERE, "cbct_oracle.h")
_LIB = os.path.join(_HERE, "libcbct_oracle.so")


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain -O2, OpenMP, no FP contraction)."""
    newest = max(os.path.getmtime(_SRC), os.path.getmtime(_HDR))
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= newest:
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-ffp-contract=off",
           "-std=c11", _SRC, "-o", tmp, "-lm"]
    subprocess.check_call(cmd)
    os.replace(tmp, _LIB)
    return _LIB


class _Geom(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
                ("dx", ctypes.c_double), ("dy", ctypes.c_double), ("dz", ctypes.c_double),
                ("nu", ctypes.c_int), ("nv", ctypes.c_int),
                ("du", ctypes.c_double), ("dv", ctypes.c_double),
                ("sad", ctypes.c_double), ("sdd", ctypes.c_double),
                ("n_views", ctypes.c_int), ("angles", ctypes.POINTER(ctypes.c_double)),
                ("step_ratio", ctypes.c_double)]


class _TV(ctypes.Structure):
    _fields_ = [("eps_tv", ctypes.c_double), ("c", ctypes.c_double),
                ("alpha", ctypes.c_double), ("rel_tol", ctypes.c_double),
                ("max_inner", ctypes.c_int), ("max_backtracks", ctypes.c_int),
                ("s0", ctypes.c_double)]


class _RofStats(ctypes.Structure):
    _fields_ = [("n_inner", ctypes.c_int), ("flags", ctypes.c_int),
                ("e_first", ctypes.c_double), ("e_last", ctypes.c_double)]


_lib = None
_D = ctypes.POINTER(ctypes.c_double)
_I = ctypes.POINTER(ctypes.c_int)


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB)
        G = ctypes.POINTER(_Geom)
        L.orc_check_geometry.argtypes = [G]
        L.orc_drho.argtypes = [G]
        L.orc_drho.restype = ctypes.c_double
        L.orc_forward_project.argtypes = [G, _D, _D]
        L.orc_forward_rays.argtypes = [G, _D, ctypes.c_int, _I, _I, _I, _D]
        L.orc_back_project.argtypes = [G, _D, _D]
        L.orc_count_terms.argtypes = [G]
        L.orc_count_terms.restype = ctypes.c_int64
        L.orc_eq6_backproject.argtypes = [G, _D, _D]
        dims = [ctypes.c_int] * 3 + [ctypes.c_double] * 3
        L.orc_tv_e1.argtypes = dims + [_D, ctypes.c_double]
        L.orc_tv_e1.restype = ctypes.c_double
        L.orc_rof_energy.argtypes = dims + [_D, _D, ctypes.c_double, ctypes.c_double, ctypes.c_double]
        L.orc_rof_energy.restype = ctypes.c_double
        L.orc_rof_gradient.argtypes = dims + [_D, _D, ctypes.c_double, ctypes.c_double,
                                              ctypes.c_double, _D]
        L.orc_rof_solve.argtypes = dims + [_D, _D, ctypes.c_double, ctypes.c_double,
                                           ctypes.POINTER(_TV), _I, ctypes.c_int, _I, ctypes.c_int,
                                           ctypes.POINTER(_RofStats)]
        L.orc_data_term.argtypes = [G, _D, _D, _D]
        L.orc_data_term.restype = ctypes.c_double
        L.orc_fbs_iteration.argtypes = [G, _D, _D, ctypes.c_double, ctypes.c_double,
                                        ctypes.POINTER(_TV), ctypes.c_int, _I, ctypes.c_int,
                                        _I, ctypes.c_int, ctypes.POINTER(_RofStats), _D]
        L.orc_power_lipschitz.argtypes = [G, ctypes.c_int]
        L.orc_power_lipschitz.restype = ctypes.c_double
        L.orc_power_lipschitz_from.argtypes = [G, _D, ctypes.c_int]
        L.orc_power_lipschitz_from.restype = ctypes.c_double
        L.orc_prolong.argtypes = [ctypes.c_int] * 3 + [_D, _D]
        _lib = L
    return _lib


def _dp(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(_D)


def _ip(a: Optional[np.ndarray]):
    if a is None:
        return None
    assert a.dtype == np.int32 and a.flags.c_contiguous
    return a.ctypes.data_as(_I)


@dataclasses.dataclass
class Geometry:
    """Circular cone-beam geometry (Fig. 1). Sizes in voxels/pixels, lengths in mm."""

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
    sad: float
    sdd: float
    angles: np.ndarray
    step_ratio: float = 0.5

    @classmethod
    def from_workload(cls, wl, level_factor: int = 1) -> "Geometry":
        f = level_factor
        return cls(wl.nx // f, wl.ny // f, wl.nz // f, wl.dx * f, wl.dy * f, wl.dz * f,
                   wl.nu, wl.nv, wl.du, wl.dv, wl.sad, wl.sdd,
                   np.ascontiguousarray(wl.angles, dtype=np.float64), wl.step_ratio)

    def coarse(self, factor: int) -> "Geometry":
        return dataclasses.replace(self, nx=self.nx // factor, ny=self.ny // factor,
                                   nz=self.nz // factor, dx=self.dx * factor,
                                   dy=self.dy * factor, dz=self.dz * factor)

    @property
    def n_views(self) -> int:
        return len(self.angles)

    @property
    def vol_shape(self):
        return (self.nx, self.ny, self.nz)

    @property
    def sino_shape(self):
        return (self.n_views, self.nv, self.nu)

    def _c(self) -> _Geom:
        self._angles_keep = np.ascontiguousarray(self.angles, dtype=np.float64)
        return _Geom(self.nx, self.ny, self.nz, self.dx, self.dy, self.dz, self.nu, self.nv,
                     self.du, self.dv, self.sad, self.sdd, len(self._angles_keep),
                     _dp(self._angles_keep), self.step_ratio)


@dataclasses.dataclass
class TVParams:
    """Sec. II.B constants: c = 0.01, alpha = 0.6, epsilon = 0.1 %."""

    eps_tv: float = 1e-5
    c: float = 0.01
    alpha: float = 0.6
    rel_tol: float = 1e-3
    max_inner: int = 50
    max_backtracks: int = 40
    s0: float = 0.0

    def _c(self) -> _TV:
        return _TV(self.eps_tv, self.c, self.alpha, self.rel_tol, self.max_inner,
                   self.max_backtracks, self.s0)


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def check_geometry(g: Geometry) -> bool:
    return lib().orc_check_geometry(ctypes.byref(g._c())) == 0


def drho(g: Geometry) -> float:
    return lib().orc_drho(ctypes.byref(g._c()))


def forward_project(g: Geometry, vol) -> np.ndarray:
    vol = _f64(vol)
    assert vol.shape == g.vol_shape
    out = np.zeros(g.sino_shape)
    rc = lib().orc_forward_project(ctypes.byref(g._c()), _dp(vol), _dp(out))
    if rc:
        raise ValueError("invalid geometry")
    return out


def forward_rays(g: Geometry, vol, view, iv, iu) -> np.ndarray:
    vol = _f64(vol)
    view = np.ascontiguousarray(view, dtype=np.int32)
    iv = np.ascontiguousarray(iv, dtype=np.int32)
    iu = np.ascontiguousarray(iu, dtype=np.int32)
    out = np.zeros(len(view))
    rc = lib().orc_forward_rays(ctypes.byref(g._c()), _dp(vol), len(view), _ip(view), _ip(iv),
                                _ip(iu), _dp(out))
    if rc:
        raise ValueError("invalid geometry")
    return out


def back_project(g: Geometry, sino) -> np.ndarray:
    sino = _f64(sino)
    assert sino.shape == g.sino_shape
    out = np.zeros(g.vol_shape)
    rc = lib().orc_back_project(ctypes.byref(g._c()), _dp(sino), _dp(out))
    if rc:
        raise ValueError("invalid geometry or out of memory")
    return out


def count_terms(g: Geometry) -> int:
    return int(lib().orc_count_terms(ctypes.byref(g._c())))


def eq6_backproject(g: Geometry, sino) -> np.ndarray:
    sino = _f64(sino)
    out = np.zeros(g.vol_shape)
    lib().orc_eq6_backproject(ctypes.byref(g._c()), _dp(sino), _dp(out))
    return out


def _dims(g: Geometry):
    return (g.nx, g.ny, g.nz, g.dx, g.dy, g.dz)


def tv_e1(g: Geometry, f, eps: float) -> float:
    f = _f64(f)
    return lib().orc_tv_e1(*_dims(g), _dp(f), eps)


def rof_energy(g: Geometry, f, gaux, lam: float, tau: float, eps: float) -> float:
    f, gaux = _f64(f), _f64(gaux)
    return lib().orc_rof_energy(*_dims(g), _dp(f), _dp(gaux), lam, tau, eps)


def rof_gradient(g: Geometry, f, gaux, lam: float, tau: float, eps: float) -> np.ndarray:
    f, gaux = _f64(f), _f64(gaux)
    d = np.zeros(g.vol_shape)
    lib().orc_rof_gradient(*_dims(g), _dp(f), _dp(gaux), lam, tau, eps, _dp(d))
    return d


@dataclasses.dataclass
class RofResult:
    f: np.ndarray
    n_inner: int
    flags: int
    e_first: float
    e_last: float
    log: np.ndarray       # step-reduction count of every accepted step


def rof_solve(g: Geometry, gaux, lam: float, tau: float, p: TVParams,
              f0=None, replay: Optional[Sequence[int]] = None) -> RofResult:
    gaux = _f64(gaux)
    f = _f64(gaux if f0 is None else f0).copy()
    log = np.zeros(max(p.max_inner, len(replay) if replay is not None else 0) + 1, dtype=np.int32)
    rep = None if replay is None else np.ascontiguousarray(replay, dtype=np.int32)
    st = _RofStats()
    tv = p._c()
    rc = lib().orc_rof_solve(*_dims(g), _dp(gaux), _dp(f), lam, tau, ctypes.byref(tv),
                             _ip(rep), 0 if rep is None else len(rep), _ip(log), len(log),
                             ctypes.byref(st))
    if rc:
        raise MemoryError("oracle ROF allocation failed")
    return RofResult(f, st.n_inner, st.flags, st.e_first, st.e_last, log[: st.n_inner].copy())


def data_term(g: Geometry, f, y) -> float:
    f, y = _f64(f), _f64(y)
    return lib().orc_data_term(ctypes.byref(g._c()), _dp(f), _dp(y), None)


def kappa(g: Geometry) -> float:
    """Gradient scale of the data term in the mean metric: 2 N_vox / (N_theta N_pix)."""
    return 2.0 * g.nx * g.ny * g.nz / (g.n_views * g.nu * g.nv)


def power_lipschitz(g: Geometry, n_iter: int = 20) -> float:
    return lib().orc_power_lipschitz(ctypes.byref(g._c()), n_iter)


def power_lipschitz_from(g: Geometry, v, n_iter: int):
    """Power iteration from start vector v; returns (L, last normalised iterate)."""
    v = _f64(v).copy()
    L = lib().orc_power_lipschitz_from(ctypes.byref(g._c()), _dp(v), n_iter)
    return L, v


def prolong(coarse) -> np.ndarray:
    coarse = _f64(coarse)
    ncx, ncy, ncz = coarse.shape
    fine = np.zeros((2 * ncx, 2 * ncy, 2 * ncz))
    lib().orc_prolong(ncx, ncy, ncz, _dp(coarse), _dp(fine))
    return fine


@dataclasses.dataclass
class IterLog:
    level: int
    e2: float
    n_inner: int
    flags: int
    e_rof_first: float
    e_rof_last: float
    steps: List[int]


def fbs_iteration_eq6(g: Geometry, y, f, lam: float, tau: float, p: TVParams, clamp: bool = True,
                      replay: Optional[Sequence[int]] = None):
    """Algorithm A1 iteration with Step 1 taken from Eq. 6 instead of P^T:
    g = f - tau kappa (voxel volume / (2 du dv)) G(P f - y). In place on f."""
    r = forward_project(g, f) - _f64(y)
    e2 = float(np.mean(r * r))
    factor = g.dx * g.dy * g.dz / (2.0 * g.du * g.dv)
    gaux = f - tau * kappa(g) * factor * eq6_backproject(g, r)
    res = rof_solve(g, gaux, lam, tau, p, replay=replay)
    f[...] = np.maximum(res.f, 0.0) if clamp else res.f
    st = _RofStats(res.n_inner, res.flags, res.e_first, res.e_last)
    return e2, st, res.log


def fbs_iteration(g: Geometry, y, f, lam: float, tau: float, p: TVParams, clamp: bool = True,
                  replay: Optional[Sequence[int]] = None):
    """One Algorithm A1 iteration in place on ``f``; returns (e2, RofStats, log)."""
    y = _f64(y)
    assert f.dtype == np.float64 and f.flags.c_contiguous
    log = np.zeros(max(p.max_inner, len(replay) if replay is not None else 0) + 1, dtype=np.int32)
    rep = None if replay is None else np.ascontiguousarray(replay, dtype=np.int32)
    st = _RofStats()
    e2 = ctypes.c_double(0.0)
    tv = p._c()
    rc = lib().orc_fbs_iteration(ctypes.byref(g._c()), _dp(y), _dp(f), lam, tau, ctypes.byref(tv),
                                 1 if clamp else 0, _ip(rep), 0 if rep is None else len(rep),
                                 _ip(log), len(log), ctypes.byref(st), ctypes.byref(e2))
    if rc:
        raise MemoryError("oracle FBS allocation failed")
    return e2.value, st, log[: st.n_inner].copy()


def round_storage(x, storage: str) -> np.ndarray:
    """Round values to a storage type and widen back to FP64, as a store and a
    later load do: first to FP32 (nearest even), then to bfloat16 (the upper
    16 bits of the FP32 pattern, nearest even) or IEEE binary16 (nearest even)."""
    x32 = np.asarray(x, dtype=np.float64).astype(np.float32)
    if storage == "f32":
        return x32.astype(np.float64)
    if storage == "fp16":
        with np.errstate(over="ignore"):   # beyond 65504 rounds to infinity, as IEEE stores do
            return x32.astype(np.float16).astype(np.float64)
    if storage == "bf16":
        u = x32.view(np.uint32).astype(np.uint64)
        u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
        return u.astype(np.uint32).view(np.float32).astype(np.float64)
    raise ValueError(storage)


def ray_ds(g: Geometry) -> np.ndarray:
    """Sample spacing along each ray, Delta rho L(u, v) / L_xy(u), per (iv, iu)
    (the same for every view): the weight every sample of P carries."""
    u = (np.arange(g.nu) - 0.5 * (g.nu - 1)) * g.du
    v = (np.arange(g.nv) - 0.5 * (g.nv - 1)) * g.dv
    lxy = np.sqrt(g.sdd ** 2 + u[None, :] ** 2)
    return drho(g) * np.sqrt(lxy ** 2 + v[:, None] ** 2) / lxy


def fbs_iteration_storage(g: Geometry, y_stored, f, lam: float, tau: float, p: TVParams, storage: str,
                          clamp: bool = True, replay: Optional[Sequence[int]] = None):
    """Algorithm A1 iteration with the projector reading a copy of f rounded to
    ``storage``, the measured sinogram already rounded (``y_stored``), and the
    residual stored, pre-weighted by the sample spacing, rounded to
    ``storage``; everything else FP64. In place on f."""
    fq = round_storage(f, storage)
    r = forward_project(g, fq) - y_stored
    e2 = float(np.mean(r * r))
    ds = ray_ds(g)[None, :, :]
    r_stored = round_storage(ds * r, storage) / ds
    gaux = f - tau * kappa(g) * back_project(g, r_stored)
    res = rof_solve(g, gaux, lam, tau, p, replay=replay)
    f[...] = np.maximum(res.f, 0.0) if clamp else res.f
    st = _RofStats(res.n_inner, res.flags, res.e_first, res.e_last)
    return e2, st, res.log


@dataclasses.dataclass
class ReconResult:
    f: np.ndarray
    taus: List[float]
    iters: List[IterLog]

    def schedule(self) -> List[List[int]]:
        """Accepted step-reduction counts of every ROF solve, in order."""
        return [it.steps for it in self.iters]


def reconstruct(g: Geometry, y, lam: float, iters: Sequence[int], p: TVParams,
                taus: Optional[Sequence[float]] = None, power_iters: int = 20,
                clamp: bool = True, f_init=None,
                replay: Optional[Sequence[Sequence[int]]] = None,
                power_iters_fine: int = 0, gradient: str = "matched", storage: str = "f32") -> ReconResult:
    """Algorithm A1 under the coarse-to-fine schedule of Sec. II.C.3.

    ``iters`` lists the FBS iterations per level, coarsest first; level l of
    L works on the grid coarsened by 2^(L-1-l) with the full detector. The
    coarsest level starts from ``f_init`` (default zero); each later level
    starts from the trilinear prolongation of the previous result. The step
    tau of each level is ``taus[l]`` when given, else 1/L from ``power_iters``
    power iterations on kappa P^T P started from ones; with
    ``power_iters_fine`` > 0, every level after the first instead runs that
    many iterations started from the prolongation of the previous level's
    last iterate. With ``storage`` other than "f32" every iteration is
    fbs_iteration_storage on the measured sinogram rounded once.
    """
    y = _f64(y)
    y_stored = round_storage(y, storage) if storage != "f32" else None
    n_levels = len(iters)
    f = None
    out_taus, logs = [], []
    k = 0
    v_eig = None
    for lev in range(n_levels):
        factor = 2 ** (n_levels - 1 - lev)
        gl = g.coarse(factor) if factor > 1 else g
        if lev == 0:
            f = np.zeros(gl.vol_shape) if f_init is None else _f64(f_init).copy()
        else:
            f = prolong(f)
        if taus is not None and taus[lev] > 0:
            tau = taus[lev]
        else:
            if lev > 0 and power_iters_fine > 0 and v_eig is not None:
                L, v_eig = power_lipschitz_from(gl, prolong(v_eig), power_iters_fine)
            else:
                L, v_eig = power_lipschitz_from(gl, np.ones(gl.vol_shape), power_iters)
            tau = 1.0 / L
        out_taus.append(tau)
        for _ in range(iters[lev]):
            rep = replay[k] if replay is not None else None
            if y_stored is not None:
                e2, st, steps = fbs_iteration_storage(gl, y_stored, f, lam, tau, p, storage, clamp, rep)
            else:
                step = fbs_iteration_eq6 if gradient == "eq6" else fbs_iteration
                e2, st, steps = step(gl, y, f, lam, tau, p, clamp, rep)
            logs.append(IterLog(lev, e2, st.n_inner, st.flags, st.e_first, st.e_last,
                                [int(s) for s in steps]))
            k += 1
    return ReconResult(f, out_taus, logs)
