"""Python binding of libcbct (include/cbct.h): argument marshalling only.

Every function here has the name of the C entry point it calls and forwards
device pointers (torch CUDA tensors), sizes and the current CUDA stream; all
computation runs in the library's CUDA kernels. There is no CPU fallback:
importing this module on a machine without the built library raises.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libcbct.so")

CBCT_MAX_LEVELS = 4
CBCT_MAX_ITERS = 512
CBCT_MAX_STEP_LOG = 8192

STATUS = {0: "CBCT_OK", 1: "CBCT_ERR_INVALID_ARG", 2: "CBCT_ERR_CUDA", 3: "CBCT_ERR_OUT_OF_MEMORY",
          4: "CBCT_ERR_WORKSPACE_TOO_SMALL", 5: "CBCT_ERR_NOT_CONVERGED", 6: "CBCT_ERR_UNSUPPORTED",
          7: "CBCT_ERR_TIMEOUT"}


class CbctError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class GeometryDesc(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
                ("dx", ctypes.c_double), ("dy", ctypes.c_double), ("dz", ctypes.c_double),
                ("nu", ctypes.c_int), ("nv", ctypes.c_int),
                ("du", ctypes.c_double), ("dv", ctypes.c_double),
                ("sad", ctypes.c_double), ("sdd", ctypes.c_double),
                ("n_views", ctypes.c_int), ("angles", ctypes.POINTER(ctypes.c_double)),
                ("step_ratio", ctypes.c_double)]


class TvParams(ctypes.Structure):
    _fields_ = [("eps_tv", ctypes.c_double), ("c", ctypes.c_double), ("alpha", ctypes.c_double),
                ("rel_tol", ctypes.c_double), ("max_inner", ctypes.c_int),
                ("max_backtracks", ctypes.c_int), ("s0", ctypes.c_double)]

    @classmethod
    def paper(cls, eps_tv: float = 1e-5, max_inner: int = 50, max_backtracks: int = 40, s0: float = 0.0):
        """Sec. II.B constants: c = 0.01, alpha = 0.6, relative tolerance 0.1 %."""
        return cls(eps_tv, 0.01, 0.6, 1e-3, max_inner, max_backtracks, s0)


class TvStats(ctypes.Structure):
    _fields_ = [("n_inner", ctypes.c_int), ("backtracks", ctypes.c_int), ("flags", ctypes.c_int),
                ("status", ctypes.c_int), ("e_first", ctypes.c_double), ("e_last", ctypes.c_double)]


class ReconParams(ctypes.Structure):
    _fields_ = [("lambda_", ctypes.c_double), ("n_levels", ctypes.c_int),
                ("iters", ctypes.c_int * CBCT_MAX_LEVELS), ("tau", ctypes.c_double * CBCT_MAX_LEVELS),
                ("power_iters", ctypes.c_int), ("clamp", ctypes.c_int), ("power_iters_fine", ctypes.c_int),
                ("gradient_mode", ctypes.c_int), ("tv", TvParams),
                ("replay", ctypes.POINTER(ctypes.c_int32)), ("replay_len", ctypes.c_int),
                ("storage", ctypes.c_int)]


class IterStats(ctypes.Structure):
    _fields_ = [("e2", ctypes.c_double), ("e_rof_first", ctypes.c_double), ("e_rof_last", ctypes.c_double),
                ("level", ctypes.c_int), ("n_inner", ctypes.c_int), ("backtracks", ctypes.c_int),
                ("flags", ctypes.c_int)]


class ReconStats(ctypes.Structure):
    _fields_ = [("tau", ctypes.c_double * CBCT_MAX_LEVELS), ("lipschitz", ctypes.c_double * CBCT_MAX_LEVELS),
                ("n_iters", ctypes.c_int), ("flags", ctypes.c_int), ("status", ctypes.c_int),
                ("n_steps", ctypes.c_int), ("iters", IterStats * CBCT_MAX_ITERS),
                ("steps", ctypes.c_int32 * CBCT_MAX_STEP_LOG)]


class ServerConfig(ctypes.Structure):
    _fields_ = [("arena_bytes", ctypes.c_size_t), ("max_resident", ctypes.c_int), ("use_graphs", ctypes.c_int),
                ("concurrency", ctypes.c_int), ("reuse_steps", ctypes.c_int)]


class ScanResult(ctypes.Structure):
    _fields_ = [("ticket", ctypes.c_uint64), ("status", ctypes.c_int32), ("graph_replay", ctypes.c_int32),
                ("recon_flags", ctypes.c_uint32), ("slot", ctypes.c_int32), ("t_submit", ctypes.c_double),
                ("t_admit", ctypes.c_double), ("t_done", ctypes.c_double), ("gpu_ms", ctypes.c_double),
                ("steps_reused", ctypes.c_int32)]


class ServerInfo(ctypes.Structure):
    _fields_ = [("arena_bytes", ctypes.c_size_t), ("bytes_in_use", ctypes.c_size_t),
                ("peak_bytes_in_use", ctypes.c_size_t), ("slots", ctypes.c_int32), ("busy_slots", ctypes.c_int32),
                ("graphs_captured", ctypes.c_int32), ("graph_failures", ctypes.c_int32),
                ("submitted", ctypes.c_int64), ("completed", ctypes.c_int64), ("evictions", ctypes.c_int64),
                ("step_reuses", ctypes.c_int64)]


_lib = None
_P = ctypes.c_void_p


def load() -> ctypes.CDLL:
    """Load libcbct.so (built in-tree by build.py). Raises if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"libcbct.so not built at {LIB_PATH}; run paper_1001_0599_gb300/build.py")
    L = ctypes.CDLL(LIB_PATH)
    st = ctypes.c_int
    L.cbct_geometry_create.argtypes = [ctypes.POINTER(GeometryDesc), ctypes.POINTER(_P)]
    L.cbct_geometry_create.restype = st
    L.cbct_geometry_destroy.argtypes = [_P]
    L.cbct_geometry_destroy.restype = None
    L.cbct_geometry_level_dims.argtypes = [_P, ctypes.c_int] + [ctypes.POINTER(ctypes.c_int)] * 3
    L.cbct_geometry_level_dims.restype = st
    L.cbct_forward_project.argtypes = [_P, _P, _P, _P]
    L.cbct_forward_project.restype = st
    L.cbct_residual.argtypes = [_P, _P, _P, _P, _P, _P, ctypes.c_size_t, _P]
    L.cbct_residual.restype = st
    L.cbct_residual_static.argtypes = [_P, _P, _P, _P, _P, _P]
    L.cbct_residual_static.restype = st
    L.cbct_back_project.argtypes = [_P, _P, _P, _P]
    L.cbct_back_project.restype = st
    L.cbct_forward_project_ex.argtypes = [_P, _P, _P, ctypes.c_int, _P]
    L.cbct_forward_project_ex.restype = st
    L.cbct_back_project_ex.argtypes = [_P, _P, ctypes.c_int, _P, _P]
    L.cbct_back_project_ex.restype = st
    L.cbct_convert.argtypes = [_P, ctypes.c_int, _P, ctypes.c_int, ctypes.c_size_t, _P]
    L.cbct_convert.restype = st
    L.cbct_eq6_gradient.argtypes = [_P, _P, _P, _P]
    L.cbct_eq6_gradient.restype = st
    L.cbct_gradient_step.argtypes = [_P, _P, _P, _P, ctypes.c_double, _P]
    L.cbct_gradient_step.restype = st
    d = ctypes.c_double
    L.cbct_tv_energy_grad.argtypes = [_P, _P, _P, d, d, d, _P, _P, _P, ctypes.c_size_t, _P]
    L.cbct_tv_energy_grad.restype = st
    L.cbct_tv_trial.argtypes = [_P, _P, _P, _P, d, d, d, d, _P, _P, ctypes.c_size_t, _P]
    L.cbct_tv_trial.restype = st
    L.cbct_tv_denoise.argtypes = [_P, _P, _P, d, d, ctypes.POINTER(TvParams), _P, ctypes.c_size_t, _P, _P]
    L.cbct_tv_denoise.restype = st
    L.cbct_check_barrier_timeout.argtypes = [_P, _P, ctypes.c_size_t, _P, _P]
    L.cbct_check_barrier_timeout.restype = st
    L.cbct_prolongate.argtypes = [ctypes.c_int] * 3 + [_P, _P, _P]
    L.cbct_prolongate.restype = st
    L.cbct_power_lipschitz.argtypes = [_P, ctypes.c_int, ctypes.c_int, _P, _P, ctypes.c_size_t, _P]
    L.cbct_power_lipschitz.restype = st
    L.cbct_workspace_size.argtypes = [_P, ctypes.POINTER(ReconParams), ctypes.POINTER(ctypes.c_size_t)]
    L.cbct_workspace_size.restype = st
    L.cbct_workspace_size_host.argtypes = [_P, ctypes.POINTER(ReconParams), ctypes.POINTER(ctypes.c_size_t)]
    L.cbct_workspace_size_host.restype = st
    L.cbct_reconstruct.argtypes = [_P, _P, _P, ctypes.POINTER(ReconParams), _P, ctypes.c_size_t, _P, _P]
    L.cbct_reconstruct.restype = st
    L.cbct_reconstruct_host.argtypes = [_P, _P, _P, ctypes.POINTER(ReconParams), _P, ctypes.c_size_t,
                                        ctypes.POINTER(ReconStats), _P]
    L.cbct_reconstruct_host.restype = st
    L.cbct_gather_bench.argtypes = [_P] + [ctypes.c_int] * 5 + [_P, _P]
    L.cbct_gather_bench.restype = st
    L.cbct_server_create.argtypes = [ctypes.POINTER(ServerConfig), ctypes.POINTER(_P)]
    L.cbct_server_create.restype = st
    L.cbct_server_destroy.argtypes = [_P]
    L.cbct_server_destroy.restype = None
    L.cbct_server_submit.argtypes = [_P, _P, ctypes.POINTER(ReconParams), _P, _P, _P, ctypes.POINTER(ctypes.c_uint64)]
    L.cbct_server_submit.restype = st
    L.cbct_server_wait.argtypes = [_P, ctypes.c_uint64, ctypes.POINTER(ScanResult)]
    L.cbct_server_wait.restype = st
    L.cbct_server_query.argtypes = [_P, ctypes.POINTER(ServerInfo)]
    L.cbct_server_query.restype = st
    L.cbct_last_error.argtypes = []
    L.cbct_last_error.restype = ctypes.c_char_p
    L.cbct_launch_count.argtypes = []
    L.cbct_launch_count.restype = ctypes.c_int64
    L.cbct_profile_enable.argtypes = [ctypes.c_int]
    L.cbct_profile_enable.restype = st
    L.cbct_profile_collect.argtypes = []
    L.cbct_profile_collect.restype = st
    L.cbct_profile_kernels.argtypes = []
    L.cbct_profile_kernels.restype = ctypes.c_int
    L.cbct_profile_name.argtypes = [ctypes.c_int]
    L.cbct_profile_name.restype = ctypes.c_char_p
    L.cbct_profile_query.argtypes = [ctypes.c_int, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_double)]
    L.cbct_profile_query.restype = st
    L.cbct_profile_query_level.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_int64),
                                           ctypes.POINTER(ctypes.c_double)]
    L.cbct_profile_query_level.restype = st
    L.cbct_profile_reset.argtypes = []
    L.cbct_profile_reset.restype = None
    _lib = L
    return L


def _check(status: int) -> None:
    if status != 0:
        raise CbctError(status, load().cbct_last_error().decode())


def _stream(stream=None) -> int:
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return s.cuda_stream


def _dev(t, name: str, dtype=None):
    """Device pointer of a contiguous CUDA tensor (None passes NULL)."""
    if t is None:
        return None
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if dtype is not None and t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}")
    return t.data_ptr()


def _f32(t, name):
    import torch
    return _dev(t, name, torch.float32)


def _f64(t, name):
    import torch
    return _dev(t, name, torch.float64)


class Geometry:
    """Owning wrapper of a cbct_geometry handle."""

    def __init__(self, handle: int, desc: GeometryDesc, angles: np.ndarray):
        self.handle = handle
        self.desc = desc
        self.angles = angles

    @property
    def vol_shape(self):
        return (self.desc.nx, self.desc.ny, self.desc.nz)

    @property
    def sino_shape(self):
        return (self.desc.n_views, self.desc.nv, self.desc.nu)

    def level_dims(self, level: int):
        return cbct_geometry_level_dims(self, level)

    def __del__(self):
        if getattr(self, "handle", None) and _lib is not None:
            _lib.cbct_geometry_destroy(self.handle)
            self.handle = None


def cbct_geometry_create(nx, ny, nz, dx, dy, dz, nu, nv, du, dv, sad, sdd, angles,
                         step_ratio: float = 0.5) -> Geometry:
    L = load()
    ang = np.ascontiguousarray(angles, dtype=np.float64)
    desc = GeometryDesc(nx, ny, nz, dx, dy, dz, nu, nv, du, dv, sad, sdd, len(ang),
                        ang.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), step_ratio)
    h = _P()
    _check(L.cbct_geometry_create(ctypes.byref(desc), ctypes.byref(h)))
    return Geometry(h.value, desc, ang)


def geometry_from_workload(wl) -> Geometry:
    return cbct_geometry_create(wl.nx, wl.ny, wl.nz, wl.dx, wl.dy, wl.dz, wl.nu, wl.nv, wl.du, wl.dv,
                                wl.sad, wl.sdd, wl.angles, wl.step_ratio)


def cbct_geometry_level_dims(geom: Geometry, level: int):
    a, b, c = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    _check(load().cbct_geometry_level_dims(geom.handle, level, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)))
    return a.value, b.value, c.value


def cbct_forward_project(geom: Geometry, vol, sino, stream=None) -> None:
    _check(load().cbct_forward_project(geom.handle, _f32(vol, "vol"), _f32(sino, "sino"), _stream(stream)))


def cbct_residual(geom: Geometry, vol, y, r, sumsq, ws, stream=None) -> None:
    _check(load().cbct_residual(geom.handle, _f32(vol, "vol"), _f32(y, "y"), _f32(r, "r"),
                                _f64(sumsq, "sumsq"), _dev(ws, "ws"), ws.numel() * ws.element_size(),
                                _stream(stream)))


def cbct_residual_static(geom: Geometry, vol, y, r, sumsq, stream=None) -> None:
    """cbct_residual without a workspace (fixed library-owned partial-sum array)."""
    _check(load().cbct_residual_static(geom.handle, _f32(vol, "vol"), _f32(y, "y"), _f32(r, "r"),
                                       _f64(sumsq, "sumsq"), _stream(stream)))


def cbct_back_project(geom: Geometry, sino, vol, stream=None) -> None:
    _check(load().cbct_back_project(geom.handle, _f32(sino, "sino"), _f32(vol, "vol"), _stream(stream)))


STORAGE = {"f32": 0, "bf16": 1, "fp16": 2}


def _storage_of(t):
    import torch
    m = {torch.float32: 0, torch.bfloat16: 1, torch.float16: 2}
    if not isinstance(t, torch.Tensor) or t.dtype not in m:
        raise TypeError("storage tensors must be float32, bfloat16 or float16")
    return m[t.dtype]


def cbct_forward_project_ex(geom: Geometry, vol, sino, stream=None) -> None:
    """P with the volume and sinogram stored as float32, bfloat16 or float16
    (both the same type; FP32 arithmetic)."""
    st = _storage_of(vol)
    if _storage_of(sino) != st:
        raise TypeError("vol and sino must share a storage type")
    _check(load().cbct_forward_project_ex(geom.handle, _dev(vol, "vol"), _dev(sino, "sino"), st, _stream(stream)))


def cbct_back_project_ex(geom: Geometry, sino, vol, stream=None) -> None:
    """Matched transpose of a float32/bfloat16/float16 sinogram into a float32 volume."""
    _check(load().cbct_back_project_ex(geom.handle, _dev(sino, "sino"), _storage_of(sino), _f32(vol, "vol"),
                                       _stream(stream)))


def cbct_convert(src, dst, stream=None) -> None:
    if src.numel() != dst.numel():
        raise ValueError("src and dst sizes differ")
    _check(load().cbct_convert(_dev(src, "src"), _storage_of(src), _dev(dst, "dst"), _storage_of(dst),
                               src.numel(), _stream(stream)))


def cbct_eq6_gradient(geom: Geometry, T, vol, stream=None) -> None:
    _check(load().cbct_eq6_gradient(geom.handle, _f32(T, "T"), _f32(vol, "vol"), _stream(stream)))


def cbct_gradient_step(geom: Geometry, r, f, g, scale: float, stream=None) -> None:
    _check(load().cbct_gradient_step(geom.handle, _f32(r, "r"), _f32(f, "f"), _f32(g, "g"), float(scale),
                                     _stream(stream)))


def cbct_tv_energy_grad(geom: Geometry, f, g, lam, tau, eps_tv, d, out, ws, stream=None) -> None:
    _check(load().cbct_tv_energy_grad(geom.handle, _f32(f, "f"), _f32(g, "g"), lam, tau, eps_tv, _f32(d, "d"),
                                      _f64(out, "out"), _dev(ws, "ws"), ws.numel() * ws.element_size(),
                                      _stream(stream)))


def cbct_tv_trial(geom: Geometry, f, d, g, s, lam, tau, eps_tv, out, ws, stream=None) -> None:
    _check(load().cbct_tv_trial(geom.handle, _f32(f, "f"), _f32(d, "d"), _f32(g, "g"), s, lam, tau, eps_tv,
                                _f64(out, "out"), _dev(ws, "ws"), ws.numel() * ws.element_size(),
                                _stream(stream)))


def cbct_tv_denoise(geom: Geometry, g, f, lam, tau, params: TvParams, ws, stats=None, stream=None) -> None:
    _check(load().cbct_tv_denoise(geom.handle, _f32(g, "g"), _f32(f, "f"), lam, tau, ctypes.byref(params),
                                  _dev(ws, "ws"), ws.numel() * ws.element_size(),
                                  _dev(stats, "stats"), _stream(stream)))


def cbct_check_barrier_timeout(geom: Geometry, ws, stats, stream=None) -> None:
    """Make the ROF kernel's bounded barrier wait expire (failure detection);
    ``stats`` (a TvStats device buffer) then reports CBCT_ERR_TIMEOUT."""
    _check(load().cbct_check_barrier_timeout(geom.handle, _dev(ws, "ws"), ws.numel() * ws.element_size(),
                                             _dev(stats, "stats"), _stream(stream)))


def cbct_prolongate(coarse, fine, stream=None) -> None:
    ncx, ncy, ncz = coarse.shape
    assert tuple(fine.shape) == (2 * ncx, 2 * ncy, 2 * ncz)
    _check(load().cbct_prolongate(ncx, ncy, ncz, _f32(coarse, "coarse"), _f32(fine, "fine"), _stream(stream)))


def cbct_power_lipschitz(geom: Geometry, level: int, n_iter: int, out, ws, stream=None) -> None:
    _check(load().cbct_power_lipschitz(geom.handle, level, n_iter, _f64(out, "out"), _dev(ws, "ws"),
                                       ws.numel() * ws.element_size(), _stream(stream)))


def make_recon_params(lam: float, iters: Sequence[int], tv: Optional[TvParams] = None,
                      taus: Optional[Sequence[float]] = None, power_iters: int = 20, clamp: bool = True,
                      replay: Optional[Sequence[Sequence[int]]] = None,
                      power_iters_fine: int = 0, gradient: str = "matched", storage: str = "f32") -> ReconParams:
    """ReconParams; ``replay`` is a list of per-iteration step-reduction lists;
    ``storage`` ("f32", "bf16", "fp16") is the type of the stored sinograms and
    of the projector's volume copy."""
    p = ReconParams()
    p.lambda_ = lam
    p.n_levels = len(iters)
    for i, n in enumerate(iters):
        p.iters[i] = int(n)
        p.tau[i] = float(taus[i]) if taus is not None else 0.0
    p.power_iters = power_iters
    p.clamp = 1 if clamp else 0
    p.power_iters_fine = power_iters_fine
    p.gradient_mode = {"matched": 0, "eq6": 1}[gradient]
    p.storage = STORAGE[storage]
    p.tv = tv if tv is not None else TvParams.paper()
    if replay is not None:
        flat = []
        for steps in replay:
            flat.append(len(steps))
            flat.extend(int(s) for s in steps)
        arr = np.ascontiguousarray(flat, dtype=np.int32)
        p._replay_keep = arr
        p.replay = arr.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))
        p.replay_len = len(arr)
    return p


def cbct_workspace_size(geom: Geometry, params: Optional[ReconParams] = None) -> int:
    n = ctypes.c_size_t()
    _check(load().cbct_workspace_size(geom.handle, ctypes.byref(params) if params is not None else None,
                                      ctypes.byref(n)))
    return n.value


def cbct_workspace_size_host(geom: Geometry, params: Optional[ReconParams] = None) -> int:
    n = ctypes.c_size_t()
    _check(load().cbct_workspace_size_host(geom.handle, ctypes.byref(params) if params is not None else None,
                                           ctypes.byref(n)))
    return n.value


def workspace(nbytes: int, device=None):
    """A 256-byte aligned device buffer of ``nbytes`` (torch allocations are)."""
    import torch
    return torch.empty(int(nbytes), dtype=torch.uint8, device=device or "cuda")


def stats_buffer(kind=ReconStats, device=None):
    import torch
    return torch.zeros(ctypes.sizeof(kind), dtype=torch.uint8, device=device or "cuda")


def read_stats(buf, kind=ReconStats):
    host = buf.cpu().numpy().tobytes()
    return kind.from_buffer_copy(host)


def cbct_reconstruct(geom: Geometry, sino, vol, params: ReconParams, ws, stats=None, stream=None) -> None:
    _check(load().cbct_reconstruct(geom.handle, _f32(sino, "sino"), _f32(vol, "vol"), ctypes.byref(params),
                                   _dev(ws, "ws"), ws.numel() * ws.element_size(), _dev(stats, "stats"),
                                   _stream(stream)))


def cbct_reconstruct_host(geom: Geometry, h_sino: np.ndarray, h_vol: np.ndarray, params: ReconParams, ws,
                          stream=None) -> ReconStats:
    """Host buffers in and out (pinned host tensors' numpy views are fine)."""
    for a, name in ((h_sino, "h_sino"), (h_vol, "h_vol")):
        if a.dtype != np.float32 or not a.flags.c_contiguous:
            raise TypeError(f"{name} must be a contiguous float32 host array")
    st = ReconStats()
    _check(load().cbct_reconstruct_host(geom.handle, h_sino.ctypes.data, h_vol.ctypes.data, ctypes.byref(params),
                                        _dev(ws, "ws"), ws.numel() * ws.element_size(), ctypes.byref(st),
                                        _stream(stream)))
    return st


def cbct_last_error() -> str:
    return load().cbct_last_error().decode()


def cbct_gather_bench(vol, n_lines: int, n_samples: int, out, stream=None) -> None:
    """cbct_gather_bench: the trilinear gather microbenchmark over the CUDA
    volume ``vol`` (nx, ny, nz); ``out`` holds n_lines * 32 floats."""
    nx, ny, nz = vol.shape
    import torch
    if out.numel() < n_lines * 32:
        raise ValueError("out must hold n_lines * 32 floats")
    _check(load().cbct_gather_bench(_dev(vol, "vol", torch.float32), nx, ny, nz, n_lines, n_samples,
                                    _dev(out, "out", torch.float32), _stream(stream)))


def cbct_launch_count() -> int:
    return int(load().cbct_launch_count())


def cbct_profile_enable(on: bool = True) -> None:
    _check(load().cbct_profile_enable(1 if on else 0))


def cbct_profile_collect() -> None:
    _check(load().cbct_profile_collect())


def cbct_profile_reset() -> None:
    load().cbct_profile_reset()


def cbct_profile_query() -> dict:
    L = load()
    out = {}
    for k in range(L.cbct_profile_kernels()):
        n, ms = ctypes.c_int64(), ctypes.c_double()
        _check(L.cbct_profile_query(k, ctypes.byref(n), ctypes.byref(ms)))
        out[L.cbct_profile_name(k).decode()] = (int(n.value), float(ms.value))
    return out


def cbct_profile_query_level(level: int) -> dict:
    """Per kernel (launches, total ms) of reconstruction launches on multigrid
    level ``level`` (0 = finest; -1: launches outside a reconstruction)."""
    L = load()
    out = {}
    for k in range(L.cbct_profile_kernels()):
        n, ms = ctypes.c_int64(), ctypes.c_double()
        _check(L.cbct_profile_query_level(k, level, ctypes.byref(n), ctypes.byref(ms)))
        out[L.cbct_profile_name(k).decode()] = (int(n.value), float(ms.value))
    return out


# ---- serving ---------------------------------------------------------------

def _host_ptr(t, name, dtype):
    """Address of a contiguous, page-locked CPU tensor."""
    import torch
    if not isinstance(t, torch.Tensor) or t.is_cuda or t.dtype != dtype:
        raise TypeError(f"{name} must be a CPU {dtype} tensor")
    if not t.is_contiguous() or not t.is_pinned():
        raise ValueError(f"{name} must be contiguous and pinned (tensor.pin_memory())")
    return t.data_ptr()


class Server:
    """Owning wrapper of a cbct_server: a native scheduler that admits scans
    into resident slots of one device arena and reconstructs them in arrival
    order, overlapping copies with computation (see include/cbct.h)."""

    def __init__(self, arena_bytes: int = 0, max_resident: int = 0, use_graphs: bool = True,
                 concurrency: int = 1, reuse_steps: bool = False):
        L = load()
        self.cfg = ServerConfig(int(arena_bytes), int(max_resident), 1 if use_graphs else 0, int(concurrency),
                                1 if reuse_steps else 0)
        h = _P()
        _check(L.cbct_server_create(ctypes.byref(self.cfg), ctypes.byref(h)))
        self.handle = h.value
        self._keep = {}

    def submit(self, geom: Geometry, params: ReconParams, h_sino, h_vol, h_stats=None) -> int:
        """Queue one scan; h_sino and h_vol are pinned float32 CPU tensors of the
        geometry's sinogram and volume shapes; returns its ticket."""
        import torch
        if tuple(h_sino.shape) != tuple(geom.sino_shape) or tuple(h_vol.shape) != tuple(geom.vol_shape):
            raise ValueError("h_sino / h_vol shapes do not match the geometry")
        stats_ptr = None
        if h_stats is not None:
            if not isinstance(h_stats, torch.Tensor) or h_stats.numel() < ctypes.sizeof(ReconStats):
                raise ValueError("h_stats must be a pinned uint8 tensor of sizeof(cbct_recon_stats) bytes")
            stats_ptr = _host_ptr(h_stats, "h_stats", torch.uint8)
        t = ctypes.c_uint64()
        _check(load().cbct_server_submit(self.handle, geom.handle, ctypes.byref(params),
                                         _host_ptr(h_sino, "h_sino", torch.float32),
                                         _host_ptr(h_vol, "h_vol", torch.float32), stats_ptr, ctypes.byref(t)))
        # the geometry, params and host buffers must outlive the scan
        self._keep[t.value] = (geom, params, h_sino, h_vol, h_stats)
        return t.value

    def wait(self, ticket: int) -> ScanResult:
        res = ScanResult()
        st = load().cbct_server_wait(self.handle, ctypes.c_uint64(ticket), ctypes.byref(res))
        self._keep.pop(ticket, None)
        _check(st)
        return res

    def query(self) -> ServerInfo:
        info = ServerInfo()
        _check(load().cbct_server_query(self.handle, ctypes.byref(info)))
        return info

    def close(self) -> None:
        if getattr(self, "handle", None):
            load().cbct_server_destroy(self.handle)
            self.handle = None
            self._keep.clear()

    def __del__(self):
        self.close()


def pinned_stats_buffer():
    """A page-locked byte buffer for one cbct_recon_stats (serving)."""
    import torch
    return torch.zeros(ctypes.sizeof(ReconStats), dtype=torch.uint8).pin_memory()


def read_host_stats(buf) -> ReconStats:
    return ReconStats.from_buffer_copy(bytes(buf.numpy().tobytes()))

