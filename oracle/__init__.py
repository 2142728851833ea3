"""FP64 CPU oracle for (locally) greedy convolutional coordinate descent.

TEST INFRASTRUCTURE ONLY: the slow, plain reference that the CUDA solver is
checked against (Moreau, Oudre & Vayatis, DICOD, ICML 2018).  Only the
tests, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline /
reference leg may import this package.  It shares no code with the CUDA
path; the arithmetic lives in ``csc_oracle.c`` (plain C, FP64,
``-ffp-contract=off``) and this module only marshals numpy arrays.

Functions and the passages they follow:
  soft_threshold   Sh(u, lambda), Sec. 2.1
  norms            ||D_k||^2, denominator of Eq. pb_coord
  crosscorr        S_{k,l}[t] = (D~_k * D_l)[t], Sec. 2.1 (Eq. beta_up)
  dtx              beta initialisation D~ * X, Alg. 1
  residual         X - sum_k Z_k * D_k, Eq. model / Sec. 2 notations
  objective        E(Z), Eq. sparse_code
  beta_fresh       beta from its definition, Sec. 2.1
  kkt              coordinate-wise optimality, Theorem A.1
  greedy_cd        Alg. 1
  locally_greedy_cd  Alg. 3 (random segments) and the segment phase schedule
  phase_count, segment_start   Sec. 2.2 segments and the phase schedule
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "csc_oracle.c")
_SO = os.path.join(_HERE, "liboracle.so")
_lib = None

_i64 = ctypes.c_longlong
_dp = ctypes.POINTER(ctypes.c_double)
_fp = ctypes.POINTER(ctypes.c_float)
_ip = ctypes.POINTER(ctypes.c_int)
_lp = ctypes.POINTER(ctypes.c_longlong)


def build(force: bool = False) -> str:
    """Compile csc_oracle.c into liboracle.so (plain gcc, no FMA contraction),
    and the 2-D variant's oracle (csc2d.py) with it."""
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + ".%d.tmp" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-std=c11", "-fPIC", "-shared",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _SO)
    from . import baseline_omp, csc2d
    csc2d.build(force)
    baseline_omp.build(force)
    return _SO


def bind(path: str):
    """Load a compiled oracle library from ``path`` and declare its signatures."""
    lib = ctypes.CDLL(path)
    lib.orc_soft_threshold.restype = ctypes.c_double
    lib.orc_soft_threshold.argtypes = [ctypes.c_double, ctypes.c_double]
    lib.orc_norms.argtypes = [_fp, ctypes.c_int, ctypes.c_int, ctypes.c_int, _dp]
    lib.orc_crosscorr.argtypes = [_fp, ctypes.c_int, ctypes.c_int, ctypes.c_int, _dp]
    lib.orc_dtx.argtypes = [_fp, _fp, ctypes.c_int, ctypes.c_int, ctypes.c_int, _i64, _dp]
    lib.orc_residual.argtypes = [_fp, _fp, _dp, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                 _i64, _dp]
    lib.orc_objective.restype = ctypes.c_double
    lib.orc_objective.argtypes = [_fp, _fp, _dp, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                  _i64, ctypes.c_double]
    lib.orc_beta_fresh.argtypes = [_fp, _fp, _dp, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                   _i64, _dp]
    lib.orc_kkt.argtypes = [_dp, _dp, _dp, ctypes.c_int, _i64, ctypes.c_double, _dp]
    lib.orc_segment_start.restype = _i64
    lib.orc_segment_start.argtypes = [_i64, ctypes.c_int, ctypes.c_int]
    lib.orc_phase_count.restype = ctypes.c_int
    lib.orc_phase_count.argtypes = [_i64, ctypes.c_int, ctypes.c_int]
    lib.orc_greedy_cd.restype = _i64
    lib.orc_greedy_cd.argtypes = [_fp, _fp, ctypes.c_int, ctypes.c_int, ctypes.c_int, _i64,
                                  ctypes.c_double, ctypes.c_double, _i64, _dp, _dp,
                                  _ip, _lp, _dp, _dp, _i64, _ip]
    lib.orc_locally_greedy_cd.restype = _i64
    lib.orc_locally_greedy_cd.argtypes = [_fp, _fp, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                          _i64, ctypes.c_double, ctypes.c_double, _i64,
                                          ctypes.c_int, ctypes.c_int, ctypes.c_ulonglong,
                                          ctypes.c_int, _dp, _dp, _ip, _lp, _dp, _dp, _i64,
                                          _ip, _lp]
    return lib


def _load():
    global _lib
    if _lib is None:
        _lib = bind(build())
    return _lib


def _f32(a):
    return np.ascontiguousarray(a, dtype=np.float32)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _p(a, t):
    return a.ctypes.data_as(t)


def soft_threshold(u: float, lam: float) -> float:
    return _load().orc_soft_threshold(float(u), float(lam))


def norms(D) -> np.ndarray:
    D = _f32(D)
    K, P, L = D.shape
    out = np.empty(K, np.float64)
    _load().orc_norms(_p(D, _fp), K, P, L, _p(out, _dp))
    return out


def crosscorr(D) -> np.ndarray:
    """S[k, l, s] = sum_u D_k[u] . D_l[u + s - (L-1)], shape [K, K, 2L-1]."""
    D = _f32(D)
    K, P, L = D.shape
    out = np.empty((K, K, 2 * L - 1), np.float64)
    _load().orc_crosscorr(_p(D, _fp), K, P, L, _p(out, _dp))
    return out


def dtx(D, X) -> np.ndarray:
    D, X = _f32(D), _f32(X)
    K, P, L = D.shape
    T = X.shape[1]
    out = np.empty((K, T - L + 1), np.float64)
    _load().orc_dtx(_p(D, _fp), _p(X, _fp), K, P, L, T, _p(out, _dp))
    return out


def lambda_max(D, X) -> float:
    """Smallest lambda for which Z = 0 is optimal: max |D~ * X| (Alg. 1 at Z = 0)."""
    return float(np.max(np.abs(dtx(D, X))))


def residual(D, X, Z) -> np.ndarray:
    D, X, Z = _f32(D), _f32(X), _f64(Z)
    K, P, L = D.shape
    T = X.shape[1]
    out = np.empty((P, T), np.float64)
    _load().orc_residual(_p(D, _fp), _p(X, _fp), _p(Z, _dp), K, P, L, T, _p(out, _dp))
    return out


def objective(D, X, Z, lam: float) -> float:
    D, X, Z = _f32(D), _f32(X), _f64(Z)
    K, P, L = D.shape
    return _load().orc_objective(_p(D, _fp), _p(X, _fp), _p(Z, _dp), K, P, L, X.shape[1],
                                 float(lam))


def beta_fresh(D, X, Z) -> np.ndarray:
    D, X, Z = _f32(D), _f32(X), _f64(Z)
    K, P, L = D.shape
    T = X.shape[1]
    out = np.empty((K, T - L + 1), np.float64)
    _load().orc_beta_fresh(_p(D, _fp), _p(X, _fp), _p(Z, _dp), K, P, L, T, _p(out, _dp))
    return out


def kkt(beta, Z, n, lam: float) -> dict:
    beta, Z, n = _f64(beta), _f64(Z), _f64(n)
    out = np.zeros(3, np.float64)
    K, Tz = Z.shape
    _load().orc_kkt(_p(beta, _dp), _p(Z, _dp), _p(n, _dp), K, Tz, float(lam), _p(out, _dp))
    return {"zero_excess": out[0], "nonzero_gap": out[1], "max_delta_z": out[2]}


def segment_start(Tz: int, M: int, m: int) -> int:
    return int(_load().orc_segment_start(Tz, M, m))


def phase_count(Tz: int, M: int, L: int) -> int:
    return int(_load().orc_phase_count(Tz, M, L))


def _trace_buffers(cap: int):
    return (np.zeros(cap, np.int32), np.zeros(cap, np.int64), np.zeros(cap, np.float64),
            np.zeros(cap, np.float64))


def _pack(Z, beta, q, conv, tr, cap, sweeps=None):
    res = {"Z": Z, "beta": beta, "n_updates": int(q), "converged": bool(conv)}
    if sweeps is not None:
        res["sweeps"] = int(sweeps)
    if cap:
        n = min(int(q), cap)
        res["trace"] = {"k": tr[0][:n].copy(), "t": tr[1][:n].copy(),
                        "z_old": tr[2][:n].copy(), "z_new": tr[3][:n].copy()}
    return res


def greedy_cd(D, X, lam: float, eps: float, max_updates: int = 10**9, trace: int = 0) -> dict:
    """Alg. 1.  Returns Z, beta (FP64), n_updates, converged (and trace)."""
    D, X = _f32(D), _f32(X)
    K, P, L = D.shape
    T = X.shape[1]
    Tz = T - L + 1
    Z = np.zeros((K, Tz), np.float64)
    beta = np.zeros((K, Tz), np.float64)
    tr = _trace_buffers(max(trace, 1))
    conv = ctypes.c_int(0)
    q = _load().orc_greedy_cd(_p(D, _fp), _p(X, _fp), K, P, L, T, float(lam), float(eps),
                              int(max_updates), _p(Z, _dp), _p(beta, _dp), _p(tr[0], _ip),
                              _p(tr[1], _lp), _p(tr[2], _dp), _p(tr[3], _dp), int(trace),
                              ctypes.byref(conv))
    if q < 0:
        raise MemoryError("oracle allocation failed")
    return _pack(Z, beta, q, conv.value, tr, trace)


def locally_greedy_cd(D, X, lam: float, eps: float, M: int, mode: str = "phase", seed: int = 0,
                      updates_per_visit: int = 0, max_updates: int = 10**12,
                      trace: int = 0) -> dict:
    """Alg. 3 (mode='random') or the segment phase schedule (mode='phase')."""
    D, X = _f32(D), _f32(X)
    K, P, L = D.shape
    T = X.shape[1]
    Tz = T - L + 1
    Z = np.zeros((K, Tz), np.float64)
    beta = np.zeros((K, Tz), np.float64)
    tr = _trace_buffers(max(trace, 1))
    conv = ctypes.c_int(0)
    sweeps = ctypes.c_longlong(0)
    q = _load().orc_locally_greedy_cd(
        _p(D, _fp), _p(X, _fp), K, P, L, T, float(lam), float(eps), int(max_updates), int(M),
        {"random": 0, "phase": 1}[mode], int(seed), int(updates_per_visit), _p(Z, _dp),
        _p(beta, _dp), _p(tr[0], _ip), _p(tr[1], _lp), _p(tr[2], _dp), _p(tr[3], _dp),
        int(trace), ctypes.byref(conv), ctypes.byref(sweeps))
    if q < 0:
        raise ValueError("oracle rejected the arguments (M must be in [1, Tz])")
    return _pack(Z, beta, q, conv.value, tr, trace, sweeps.value)
