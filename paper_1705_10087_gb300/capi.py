"""Thin Python binding of the C ABI in include/csc.h (ctypes).

The functions carry the C names and only marshal arguments: arrays may be
torch tensors (CUDA or CPU) or numpy arrays and are passed as raw pointers;
every computation runs in libcsc.so.  There is no fallback: if the library
is missing, loading it raises.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

CSC_OK = 0
CSC_NOT_CONVERGED = 1
CSC_EINVAL = -1
CSC_ENOMEM = -2
CSC_ECUDA = -3
CSC_ETIMEOUT = -4
CSC_ESTATE = -5


class csc_opts(ctypes.Structure):
    _fields_ = [("segments", ctypes.c_int32), ("updates_per_visit", ctypes.c_int32),
                ("max_resyncs", ctypes.c_int32), ("sweeps_per_poll", ctypes.c_int32),
                ("max_sweeps", ctypes.c_int32), ("time_kernels", ctypes.c_int32),
                ("segment_width", ctypes.c_int32), ("init_mode", ctypes.c_int32),
                ("launch_mode", ctypes.c_int32), ("threads_per_segment", ctypes.c_int32)]


class csc_stats(ctypes.Structure):
    _fields_ = [("updates", ctypes.c_int64), ("sweeps", ctypes.c_int64),
                ("segments", ctypes.c_int32), ("phases", ctypes.c_int32),
                ("resyncs", ctypes.c_int32), ("converged", ctypes.c_int32),
                ("objective", ctypes.c_double), ("max_drift", ctypes.c_double),
                ("kkt_zero_excess", ctypes.c_double), ("kkt_nonzero_gap", ctypes.c_double),
                ("max_delta_z", ctypes.c_double), ("solve_ms", ctypes.c_double),
                ("phase_ms", ctypes.c_double), ("phase_launches", ctypes.c_int64),
                ("visits", ctypes.c_int64), ("kernel_launches", ctypes.c_int64),
                ("drift_resyncs", ctypes.c_int64), ("resync_ms", ctypes.c_double),
                ("objective_ms", ctypes.c_double)]

    def as_dict(self) -> dict:
        return {name: getattr(self, name) for name, _ in self._fields_}


class csc_tune_result(ctypes.Structure):
    _fields_ = [("segment_width", ctypes.c_int32), ("updates_per_visit", ctypes.c_int32),
                ("phases", ctypes.c_int32), ("candidates", ctypes.c_int32),
                ("best_ms", ctypes.c_double), ("default_ms", ctypes.c_double),
                ("threads_per_segment", ctypes.c_int32)]

    def as_dict(self) -> dict:
        return {name: getattr(self, name) for name, _ in self._fields_}


class csc_server_opts(ctypes.Structure):
    _fields_ = [("hbm_budget_bytes", ctypes.c_int64), ("sweeps_per_step", ctypes.c_int32),
                ("max_resyncs", ctypes.c_int32), ("max_active", ctypes.c_int32),
                ("reserved", ctypes.c_int32 * 3)]


class csc_request_info(ctypes.Structure):
    _fields_ = [("state", ctypes.c_int32), ("dict", ctypes.c_int32), ("T", ctypes.c_int64),
                ("lambda_", ctypes.c_double), ("lambda_max", ctypes.c_double),
                ("objective", ctypes.c_double), ("max_delta_z", ctypes.c_double),
                ("resyncs", ctypes.c_int32), ("converged", ctypes.c_int32),
                ("rounds", ctypes.c_int64), ("device_bytes", ctypes.c_int64),
                ("t_submit", ctypes.c_double), ("t_admit", ctypes.c_double),
                ("t_done", ctypes.c_double)]

    def as_dict(self) -> dict:
        d = {name: getattr(self, name) for name, _ in self._fields_}
        d["lambda"] = d.pop("lambda_")
        return d


CSC_REQ_QUEUED, CSC_REQ_ACTIVE, CSC_REQ_DONE = 0, 1, 2


class csc2d_stats(ctypes.Structure):
    _fields_ = [("updates", ctypes.c_int64), ("sweeps", ctypes.c_int64),
                ("bands", ctypes.c_int32), ("col_blocks", ctypes.c_int32),
                ("phases", ctypes.c_int32), ("resyncs", ctypes.c_int32),
                ("converged", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("objective", ctypes.c_double), ("max_delta_z", ctypes.c_double),
                ("solve_ms", ctypes.c_double), ("kernel_launches", ctypes.c_int64)]

    def as_dict(self) -> dict:
        return {name: getattr(self, name) for name, _ in self._fields_}


class csc_shard_plan(ctypes.Structure):
    _fields_ = [("T", ctypes.c_int64), ("Tz", ctypes.c_int64), ("L", ctypes.c_int32),
                ("M", ctypes.c_int32), ("phases", ctypes.c_int32), ("world", ctypes.c_int32),
                ("rank", ctypes.c_int32), ("seg_first", ctypes.c_int32),
                ("seg_count", ctypes.c_int32), ("col_first", ctypes.c_int64),
                ("col_count", ctypes.c_int64), ("halo_left", ctypes.c_int64),
                ("halo_right", ctypes.c_int64), ("x_first", ctypes.c_int64),
                ("x_count", ctypes.c_int64)]

    def as_dict(self) -> dict:
        return {name: getattr(self, name) for name, _ in self._fields_}


class CscError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"csc error {status}: {message}")
        self.status = status


_lib = None
_vp = ctypes.c_void_p
_i64 = ctypes.c_int64


def library_path() -> str:
    return _build.LIB


def load(path: str | None = None):
    """Load libcsc.so (build it first with build.build()); raises if absent."""
    global _lib
    if _lib is not None and path is None:
        return _lib
    path = path or _build.LIB
    if not os.path.exists(path):
        raise OSError(f"{path} is not built: run paper_1705_10087_gb300.build.build()")
    lib = ctypes.CDLL(path)
    lib.csc_default_opts.argtypes = [ctypes.POINTER(csc_opts)]
    lib.csc_default_opts.restype = None
    lib.csc_setup.argtypes = [ctypes.POINTER(_vp), _vp, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                              ctypes.POINTER(csc_opts), _vp]
    lib.csc_init.argtypes = [_vp, _vp, _i64, ctypes.c_double, _vp]
    lib.csc_solve.argtypes = [_vp, ctypes.c_double, _i64, _vp, ctypes.POINTER(ctypes.c_double),
                              ctypes.POINTER(csc_stats)]
    lib.csc_destroy.argtypes = [_vp]
    lib.csc_lambda_max.argtypes = [_vp, ctypes.POINTER(ctypes.c_double)]
    lib.csc_get_beta.argtypes = [_vp, _vp]
    lib.csc_get_dtd.argtypes = [_vp, _vp, _vp]
    lib.csc_objective.argtypes = [_vp, _vp, ctypes.POINTER(ctypes.c_double)]
    lib.csc_kkt.argtypes = [_vp, _vp, _vp]
    lib.csc_get_trace.argtypes = [_vp, _i64, _vp, _vp, _vp, ctypes.POINTER(_i64),
                                  ctypes.POINTER(ctypes.c_double)]
    lib.csc_plan.argtypes = [_i64, ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_int),
                             ctypes.POINTER(ctypes.c_int), _vp]
    lib.csc_kernel_launches.argtypes = [_vp, ctypes.POINTER(_i64)]
    lib.csc_init_time.argtypes = [_vp, ctypes.POINTER(ctypes.c_double)]
    lib.csc_check_wait_timeout.argtypes = [_i64]
    lib.csc_objective_noalloc.argtypes = [_vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, _vp,
                                          _i64, _vp, ctypes.c_double, _vp, _vp]
    lib.csc_init_batch.argtypes = [_vp, _vp, _vp, ctypes.c_int, _vp, _vp]
    lib.csc_set_lambda.argtypes = [_vp, _vp]
    lib.csc_lambda_max_batch.argtypes = [_vp, _vp]
    lib.csc_get_objectives.argtypes = [_vp, _vp]
    lib.csc_autotune.argtypes = [_vp, ctypes.c_double, _i64, ctypes.POINTER(csc_tune_result)]
    lib.csc_server_create.argtypes = [ctypes.POINTER(_vp), ctypes.POINTER(csc_server_opts)]
    lib.csc_server_add_dictionary.argtypes = [_vp, _vp, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                              ctypes.c_int32, ctypes.c_int32,
                                              ctypes.POINTER(ctypes.c_int)]
    lib.csc_server_submit.argtypes = [_vp, ctypes.c_int, _vp, _i64, ctypes.c_double,
                                      ctypes.c_double, ctypes.POINTER(_i64)]
    lib.csc_server_step.argtypes = [_vp, ctypes.POINTER(ctypes.c_int),
                                    ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)]
    lib.csc_server_info.argtypes = [_vp, _i64, ctypes.POINTER(csc_request_info)]
    lib.csc_server_completed.argtypes = [_vp, _vp, ctypes.c_int, ctypes.POINTER(ctypes.c_int)]
    lib.csc_server_fetch.argtypes = [_vp, _i64, _vp, ctypes.POINTER(csc_request_info)]
    lib.csc_server_memory.argtypes = [_vp, ctypes.POINTER(_i64), ctypes.POINTER(_i64),
                                      ctypes.POINTER(_i64)]
    lib.csc_server_kernel_launches.argtypes = [_vp, ctypes.POINTER(_i64)]
    lib.csc_server_destroy.argtypes = [_vp]
    lib.csc_shard_plan_make.argtypes = [_i64, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                        ctypes.c_int, ctypes.POINTER(csc_shard_plan)]
    lib.csc_shard_init.argtypes = [_vp, ctypes.POINTER(csc_shard_plan), _vp, ctypes.c_double]
    lib.csc_shard_phase.argtypes = [_vp, ctypes.c_int, ctypes.c_double]
    for name in ("csc_shard_halo_out", "csc_shard_halo_in", "csc_shard_z_out",
                 "csc_shard_z_in"):
        getattr(lib, name).argtypes = [_vp, _vp, _vp]
    lib.csc_shard_updates.argtypes = [_vp, ctypes.POINTER(_i64)]
    lib.csc_shard_resync.argtypes = [_vp, ctypes.c_double, ctypes.POINTER(ctypes.c_double)]
    lib.csc_shard_objective.argtypes = [_vp, ctypes.POINTER(ctypes.c_double)]
    lib.csc_shard_get_z.argtypes = [_vp, _vp]
    lib.csc2d_plan.argtypes = [_i64, ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_int),
                               ctypes.POINTER(ctypes.c_int), _vp]
    lib.csc2d_solve.argtypes = [_vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, _vp,
                                _i64, _i64, ctypes.c_double, ctypes.c_double, _i64, ctypes.c_int,
                                ctypes.c_int, ctypes.c_int, _vp, ctypes.POINTER(ctypes.c_double),
                                ctypes.POINTER(csc2d_stats), _vp]
    lib.csc_last_error_string.argtypes = []
    lib.csc_last_error_string.restype = ctypes.c_char_p
    for name in ("csc_setup", "csc_init", "csc_solve", "csc_destroy", "csc_lambda_max",
                 "csc_get_beta", "csc_get_dtd", "csc_objective", "csc_get_trace", "csc_plan",
                 "csc_kernel_launches", "csc_init_time", "csc_objective_noalloc", "csc_init_batch",
                 "csc_set_lambda", "csc_lambda_max_batch", "csc_get_objectives",
                 "csc_autotune", "csc_server_create", "csc_server_add_dictionary",
                 "csc_server_submit", "csc_server_step", "csc_server_info", "csc_server_fetch",
                 "csc_server_completed", "csc_check_wait_timeout", "csc_kkt",
                 "csc_server_memory", "csc_server_kernel_launches", "csc_server_destroy",
                 "csc_shard_plan_make", "csc_shard_init", "csc_shard_phase",
                 "csc_shard_halo_out", "csc_shard_halo_in", "csc_shard_z_out",
                 "csc_shard_z_in", "csc_shard_updates", "csc_shard_resync",
                 "csc_shard_objective", "csc_shard_get_z", "csc2d_plan", "csc2d_solve"):
        getattr(lib, name).restype = ctypes.c_int
    if path == _build.LIB:
        _lib = lib
    return lib


def csc_last_error_string() -> str:
    return load().csc_last_error_string().decode()


def _check(status: int) -> int:
    if status < 0:
        raise CscError(status, csc_last_error_string())
    return status


def _ptr(a, writable: bool = False):
    """Raw pointer of a float32 contiguous torch tensor or numpy array."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        if a.dtype != np.float32 or not a.flags.c_contiguous:
            raise TypeError("numpy arrays must be C-contiguous float32")
        if writable and not a.flags.writeable:
            raise TypeError("output array is read-only")
        return a.ctypes.data
    import torch
    if isinstance(a, torch.Tensor):
        if a.dtype != torch.float32 or not a.is_contiguous():
            raise TypeError("tensors must be contiguous float32")
        return a.data_ptr()
    raise TypeError(f"unsupported array type {type(a)!r}")


class Handle(_vp):
    """A csc handle (an opaque C pointer) that remembers the sizes (K, P, L) of
    its dictionary, so that the binding can check array shapes before it
    passes their pointers on."""
    K = P = L = None
    Tz = None  # columns of the current problem (set by csc_init / csc_init_batch)


def _shape(a):
    return tuple(int(x) for x in a.shape)


def _device_of(a):
    """("cuda", index) for a CUDA tensor, ("cpu", None) for anything else."""
    dev = getattr(a, "device", None)
    if dev is not None and getattr(dev, "type", "cpu") == "cuda":
        return ("cuda", dev.index)
    return ("cpu", None)


def _check_signal(h, X, what: str = "X"):
    if len(X.shape) != 2:
        raise ValueError(f"{what} must be [P, T]")
    if h is not None and getattr(h, "P", None) is not None and int(X.shape[0]) != h.P:
        raise ValueError(f"{what} has {int(X.shape[0])} channels, the dictionary {h.P}")


def _check_z(h, Z, Tz: int, what: str = "Z"):
    if Z is None or h is None or getattr(h, "K", None) is None:
        return
    if int(np.prod(_shape(Z))) != h.K * Tz:
        raise ValueError(f"{what} must hold K * Tz = {h.K} * {Tz} values, got shape "
                         f"{_shape(Z)}")


def _stream(stream):
    if stream is not None:
        return stream if isinstance(stream, int) else stream.cuda_stream
    import torch
    return torch.cuda.current_stream().cuda_stream


def csc_default_opts() -> csc_opts:
    """The library's default options (every field as include/csc.h documents)."""
    o = csc_opts()
    load().csc_default_opts(ctypes.byref(o))
    return o


def make_opts(segments: int = 0, updates_per_visit: int = 0, max_resyncs: int = -1,
              sweeps_per_poll: int = 0, max_sweeps: int = 0, time_kernels: int = 0,
              segment_width: int = 0, init_mode: int = 0, launch_mode: int = 0,
              threads_per_segment: int = 0) -> csc_opts:
    o = csc_default_opts()
    o.segments, o.updates_per_visit = segments, updates_per_visit
    o.max_resyncs, o.sweeps_per_poll, o.max_sweeps = max_resyncs, sweeps_per_poll, max_sweeps
    o.time_kernels, o.segment_width, o.init_mode = time_kernels, segment_width, init_mode
    o.launch_mode = launch_mode
    o.threads_per_segment = threads_per_segment
    return o


def csc_setup(D, opts: csc_opts | None = None, stream=None, handle=None):
    """D [K,P,L] float32 -> handle (a ctypes c_void_p); re-uses ``handle`` if given."""
    if len(D.shape) != 3:
        raise ValueError("D must be [K, P, L]")
    K, P, L = (int(x) for x in D.shape)
    h = handle if handle is not None else Handle()
    _check(load().csc_setup(ctypes.byref(h), _ptr(D), K, P, L,
                            ctypes.byref(opts) if opts is not None else None, _stream(stream)))
    if isinstance(h, Handle):
        h.K, h.P, h.L, h.Tz = K, P, L, None  # a new setup invalidates the problem
    return h


def csc_init(h, X, lam: float, Z0=None) -> None:
    _check_signal(h, X)
    if getattr(h, "L", None) is not None:
        _check_z(h, Z0, int(X.shape[1]) - h.L + 1, "Z0")
    _check(load().csc_init(h, _ptr(X), int(X.shape[1]), float(lam), _ptr(Z0)))
    if isinstance(h, Handle) and h.L is not None:
        h.Tz = int(X.shape[1]) - h.L + 1


def csc_init_batch(h, X, T, lam, Z0=None) -> None:
    """X [P, sum T] (signals concatenated in time); T and lam: one entry per signal."""
    Ta = np.ascontiguousarray(np.asarray(T, dtype=np.int64).reshape(-1))
    la = np.ascontiguousarray(np.asarray(lam, dtype=np.float64).reshape(-1))
    if la.shape != Ta.shape:
        raise ValueError("T and lam need one entry per signal")
    _check_signal(h, X)
    if int(Ta.sum()) != int(X.shape[1]):
        raise ValueError("X must hold sum(T) samples per channel")
    if getattr(h, "L", None) is not None:
        _check_z(h, Z0, int(Ta.sum()) - h.L + 1, "Z0")
    _check(load().csc_init_batch(h, _ptr(X), Ta.ctypes.data, int(Ta.size), la.ctypes.data,
                                 _ptr(Z0)))
    if isinstance(h, Handle) and h.L is not None:
        h.Tz = int(Ta.sum()) - h.L + 1


def csc_set_lambda(h, lam) -> None:
    la = np.ascontiguousarray(np.asarray(lam, dtype=np.float64).reshape(-1))
    _check(load().csc_set_lambda(h, la.ctypes.data))


def csc_lambda_max_batch(h, n: int) -> np.ndarray:
    out = np.zeros(n, np.float64)
    _check(load().csc_lambda_max_batch(h, out.ctypes.data))
    return out


def csc_get_objectives(h, n: int) -> np.ndarray:
    out = np.zeros(n, np.float64)
    _check(load().csc_get_objectives(h, out.ctypes.data))
    return out


def csc_autotune(h, tol: float, max_updates: int = 1 << 62) -> dict:
    r = csc_tune_result()
    _check(load().csc_autotune(h, float(tol), int(max_updates), ctypes.byref(r)))
    return r.as_dict()


def csc_solve(h, tol: float, max_updates: int = 1 << 62, Z_out=None):
    """Returns (status, objective, stats dict)."""
    if getattr(h, "Tz", None) is not None:
        _check_z(h, Z_out, h.Tz, "Z_out")
    obj = ctypes.c_double(0.0)
    st = csc_stats()
    status = _check(load().csc_solve(h, float(tol), int(max_updates), _ptr(Z_out, True),
                                     ctypes.byref(obj), ctypes.byref(st)))
    return status, obj.value, st.as_dict()


def csc_destroy(h) -> None:
    _check(load().csc_destroy(h))


def csc_lambda_max(h) -> float:
    v = ctypes.c_double(0.0)
    _check(load().csc_lambda_max(h, ctypes.byref(v)))
    return v.value


def csc_get_beta(h, out) -> None:
    if getattr(h, "Tz", None) is not None:
        _check_z(h, out, h.Tz, "beta_out")
    _check(load().csc_get_beta(h, _ptr(out, True)))


def csc_get_dtd(h, dtd_out=None, norms_out=None) -> None:
    _check(load().csc_get_dtd(h, _ptr(dtd_out, True), _ptr(norms_out, True)))


def csc_objective(h, Z) -> float:
    if getattr(h, "Tz", None) is not None:
        _check_z(h, Z, h.Tz)
    v = ctypes.c_double(0.0)
    _check(load().csc_objective(h, _ptr(Z), ctypes.byref(v)))
    return v.value


def csc_kkt(h, Z) -> dict:
    """Optimality report of Z (Theorem A.1) for the handle's X and lambda."""
    if getattr(h, "Tz", None) is not None:
        _check_z(h, Z, h.Tz)
    out = np.zeros(3, np.float64)
    _check(load().csc_kkt(h, _ptr(Z), out.ctypes.data))
    return {"zero_excess": float(out[0]), "nonzero_gap": float(out[1]),
            "max_delta_z": float(out[2])}


def csc_get_trace(h, cap: int = 1 << 16) -> dict:
    upd = np.zeros(cap, np.int64)
    dec = np.zeros(cap, np.float64)
    tns = np.zeros(cap, np.int64)
    n = _i64(0)
    e0 = ctypes.c_double(0.0)
    _check(load().csc_get_trace(h, cap, upd.ctypes.data, dec.ctypes.data, tns.ctypes.data,
                                ctypes.byref(n), ctypes.byref(e0)))
    m = min(int(n.value), cap)
    return {"updates": upd[:m], "decrease": dec[:m], "t_ns": tns[:m], "n": int(n.value),
            "E_start": e0.value}


def csc_objective_noalloc(D, X, Z, lam: float, out=None, stream=None) -> float:
    """E(Z) through the allocation-free entry point; D, X, Z must be CUDA tensors.
    ``out`` may be a one-element float64 CUDA tensor to receive E on the device."""
    if len(D.shape) != 3:
        raise ValueError("D must be [K, P, L]")
    K, P, L = (int(x) for x in D.shape)
    if _shape(X)[:1] != (P,) or len(X.shape) != 2:
        raise ValueError(f"X must be [P={P}, T], got shape {_shape(X)}")
    T = int(X.shape[1])
    if T < L:
        raise ValueError(f"X has T = {T} < L = {L} samples")
    if _shape(Z) != (K, T - L + 1):
        raise ValueError(f"Z must be [K={K}, T-L+1={T - L + 1}], got shape {_shape(Z)}")
    devs = {_device_of(a) for a in (D, X, Z) + (() if out is None else (out,))}
    if len(devs) != 1 or next(iter(devs))[0] != "cuda":
        raise ValueError("D, X, Z (and out) must be CUDA tensors on one device")
    if out is None:
        v = ctypes.c_double(0.0)
        _check(load().csc_objective_noalloc(_ptr(D), K, P, L, _ptr(X), int(X.shape[1]), _ptr(Z),
                                            float(lam), ctypes.addressof(v), _stream(stream)))
        return v.value
    import torch
    if out.dtype != torch.float64 or out.numel() != 1 or not out.is_cuda:
        raise TypeError("out must be a one-element float64 CUDA tensor")
    _check(load().csc_objective_noalloc(_ptr(D), K, P, L, _ptr(X), int(X.shape[1]), _ptr(Z),
                                        float(lam), out.data_ptr(), _stream(stream)))
    return float(out.item())


def csc_init_time(h) -> float:
    """Device ms of the last csc_init's beta0 kernel (opts.time_kernels = 1), else -1."""
    v = ctypes.c_double(0.0)
    _check(load().csc_init_time(h, ctypes.byref(v)))
    return v.value


def csc_kernel_launches(h) -> int:
    v = _i64(0)
    _check(load().csc_kernel_launches(h, ctypes.byref(v)))
    return v.value


def csc_check_wait_timeout(polls: int) -> int:
    """Raw status of the bounded-wait check (CSC_ETIMEOUT expected), no raise."""
    return int(load().csc_check_wait_timeout(int(polls)))


def csc_plan(Tz: int, L: int, M: int = 0):
    """Host-only schedule: returns (M, phases, starts[M+1])."""
    Mo = ctypes.c_int(0)
    c = ctypes.c_int(0)
    _check(load().csc_plan(int(Tz), int(L), int(M), ctypes.byref(Mo), ctypes.byref(c), None))
    starts = np.zeros(Mo.value + 1, np.int64)
    _check(load().csc_plan(int(Tz), int(L), Mo.value, None, None, starts.ctypes.data))
    return Mo.value, c.value, starts


# ------------------------------------------------------------------ server

def csc_server_create(hbm_budget_bytes: int = 0, sweeps_per_step: int = 0,
                      max_resyncs: int = -1, max_active: int = 0):
    o = csc_server_opts()
    o.hbm_budget_bytes, o.sweeps_per_step = hbm_budget_bytes, sweeps_per_step
    o.max_resyncs, o.max_active = max_resyncs, max_active
    s = _vp()
    _check(load().csc_server_create(ctypes.byref(s), ctypes.byref(o)))
    return s


def csc_server_add_dictionary(s, D, segment_width: int = 0, updates_per_visit: int = 0) -> int:
    K, P, L = (int(x) for x in D.shape)
    d = ctypes.c_int(0)
    _check(load().csc_server_add_dictionary(s, _ptr(D), K, P, L, segment_width,
                                            updates_per_visit, ctypes.byref(d)))
    return d.value


def csc_server_submit(s, dict_id: int, X, lam: float, tol: float) -> int:
    """lam > 0: absolute lambda; lam < 0: |lam| * lambda_max of X."""
    r = _i64(0)
    _check(load().csc_server_submit(s, int(dict_id), _ptr(X), int(X.shape[1]), float(lam),
                                    float(tol), ctypes.byref(r)))
    return r.value


def csc_server_step(s):
    """One scheduling round -> (active, queued, finished in this round)."""
    a, q, d = ctypes.c_int(0), ctypes.c_int(0), ctypes.c_int(0)
    _check(load().csc_server_step(s, ctypes.byref(a), ctypes.byref(q), ctypes.byref(d)))
    return a.value, q.value, d.value


def csc_server_completed(s, cap: int = 4096) -> list:
    """Ids of the requests that finished since the previous call."""
    buf = np.zeros(cap, np.int64)
    n = ctypes.c_int(0)
    _check(load().csc_server_completed(s, buf.ctypes.data, cap, ctypes.byref(n)))
    return [int(x) for x in buf[:n.value]]


def csc_server_info(s, req: int) -> dict:
    info = csc_request_info()
    _check(load().csc_server_info(s, int(req), ctypes.byref(info)))
    return info.as_dict()


def csc_server_fetch(s, req: int, Z_out=None) -> dict:
    info = csc_request_info()
    _check(load().csc_server_fetch(s, int(req), _ptr(Z_out, True), ctypes.byref(info)))
    return info.as_dict()


def csc_server_memory(s):
    a, b, c = _i64(0), _i64(0), _i64(0)
    _check(load().csc_server_memory(s, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)))
    return {"pool_bytes": a.value, "in_use": b.value, "peak": c.value}


def csc_server_kernel_launches(s) -> int:
    v = _i64(0)
    _check(load().csc_server_kernel_launches(s, ctypes.byref(v)))
    return v.value


def csc_server_destroy(s) -> None:
    _check(load().csc_server_destroy(s))


# ------------------------------------------------------------------ shards

def csc_shard_plan_make(T: int, L: int, M: int, world: int, rank: int) -> dict:
    """Host-only plan of rank `rank` of `world` (include/csc_shard.h)."""
    p = csc_shard_plan()
    _check(load().csc_shard_plan_make(int(T), int(L), int(M), int(world), int(rank),
                                      ctypes.byref(p)))
    return p.as_dict()


def _plan_struct(plan: dict) -> csc_shard_plan:
    p = csc_shard_plan()
    for name, _ in p._fields_:
        setattr(p, name, int(plan[name]))
    return p


def _check_block(h, a, width: int, what: str):
    if width == 0 or a is None:
        return
    if getattr(h, "K", None) is not None and _shape(a) != (h.K, width):
        raise ValueError(f"{what} must be [K={h.K}, {width}], got shape {_shape(a)}")


def csc_shard_init(h, plan: dict, X, lam: float) -> None:
    """X: this rank's samples [P, plan['x_count']]."""
    _check_signal(h, X)
    if int(X.shape[1]) != int(plan["x_count"]):
        raise ValueError(f"X must hold x_count = {plan['x_count']} samples per channel")
    p = _plan_struct(plan)
    _check(load().csc_shard_init(h, ctypes.byref(p), _ptr(X), float(lam)))
    if isinstance(h, Handle):
        h.Tz = None
        h.shard = dict(plan)


def csc_shard_phase(h, p: int, tol: float) -> None:
    _check(load().csc_shard_phase(h, int(p), float(tol)))


def _blocks(h, name, a, b):
    sh = getattr(h, "shard", None)
    if sh is not None:
        _check_block(h, a, int(sh["halo_left"]), f"{name} left block")
        _check_block(h, b, int(sh["halo_right"]), f"{name} right block")
    return _ptr(a, True) if a is not None else None, _ptr(b, True) if b is not None else None


def csc_shard_halo_out(h, to_left, to_right) -> None:
    _check(load().csc_shard_halo_out(h, *_blocks(h, "halo_out", to_left, to_right)))


def csc_shard_halo_in(h, from_left, from_right) -> None:
    _check(load().csc_shard_halo_in(h, *_blocks(h, "halo_in", from_left, from_right)))


def csc_shard_z_out(h, to_left, to_right) -> None:
    _check(load().csc_shard_z_out(h, *_blocks(h, "z_out", to_left, to_right)))


def csc_shard_z_in(h, from_left, from_right) -> None:
    _check(load().csc_shard_z_in(h, *_blocks(h, "z_in", from_left, from_right)))


def csc_shard_updates(h) -> int:
    v = _i64(0)
    _check(load().csc_shard_updates(h, ctypes.byref(v)))
    return v.value


def csc_shard_resync(h, tol: float) -> float:
    v = ctypes.c_double(0.0)
    _check(load().csc_shard_resync(h, float(tol), ctypes.byref(v)))
    return v.value


def csc_shard_objective(h) -> float:
    v = ctypes.c_double(0.0)
    _check(load().csc_shard_objective(h, ctypes.byref(v)))
    return v.value


def csc_shard_get_z(h, out) -> None:
    sh = getattr(h, "shard", None)
    if sh is not None and getattr(h, "K", None) is not None:
        if int(np.prod(_shape(out))) != h.K * int(sh["col_count"]):
            raise ValueError("Z_out must hold K * col_count values")
    _check(load().csc_shard_get_z(h, _ptr(out, True)))


# ------------------------------------------------------------------ images (2-D)

def csc2d_plan(Hz: int, h: int, M: int = 0):
    """Host-only band schedule: (M, phases, starts[M+1])."""
    Mo, c = ctypes.c_int(0), ctypes.c_int(0)
    _check(load().csc2d_plan(int(Hz), int(h), int(M), ctypes.byref(Mo), ctypes.byref(c), None))
    starts = np.zeros(Mo.value + 1, np.int64)
    _check(load().csc2d_plan(int(Hz), int(h), Mo.value, None, None, starts.ctypes.data))
    return Mo.value, c.value, starts


def csc2d_solve(D, X, lam: float, tol: float, max_updates: int = 1 << 62, M: int = 0,
                N: int = 0, updates_per_visit: int = 0, Z_out=None, stream=None):
    """D [K,P,h,w], X [P,H,W] -> (status, objective, stats dict)."""
    if len(D.shape) != 4 or len(X.shape) != 3:
        raise ValueError("D must be [K, P, h, w] and X [P, H, W]")
    K, P, h, w = (int(x) for x in D.shape)
    if int(X.shape[0]) != P:
        raise ValueError(f"X has {int(X.shape[0])} channels, D {P}")
    H, W = int(X.shape[1]), int(X.shape[2])
    if Z_out is not None and int(np.prod(_shape(Z_out))) != K * (H - h + 1) * (W - w + 1):
        raise ValueError("Z_out must hold K * (H-h+1) * (W-w+1) values")
    obj = ctypes.c_double(0.0)
    st = csc2d_stats()
    status = _check(load().csc2d_solve(_ptr(D), K, P, h, w, _ptr(X), H, W, float(lam),
                                       float(tol), int(max_updates), int(M), int(N),
                                       int(updates_per_visit), _ptr(Z_out, True),
                                       ctypes.byref(obj), ctypes.byref(st), _stream(stream)))
    return status, obj.value, st.as_dict()
