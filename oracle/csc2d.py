"""FP64 CPU oracle of the 2-D variant: images cut into row bands (one axis).

TEST INFRASTRUCTURE ONLY, like the rest of this package: the arithmetic lives
in ``csc2d_oracle.c`` (plain C, FP64, ``-ffp-contract=off``) and this module
only marshals numpy arrays.  The paper's conclusion names cutting images along
a single direction as the way to keep its 1-D analysis; every definition is
that of Sec. 2.1 with 2-D lags.

Functions and the passages they follow (2-D forms):
  norms            ||D_k||^2, denominator of Eq. pb_coord
  crosscorr        S_{k,l}[a, b], Sec. 2.1 (Eq. beta_up)
  dtx              beta initialisation D~ * X, Alg. 1
  residual         X - sum_k Z_k * D_k
  objective        E(Z), Eq. sparse_code
  beta_fresh       beta from its definition, Sec. 2.1
  greedy_cd        Alg. 1
  locally_greedy_cd  Alg. 3 on row bands (random bands) and the band phase schedule
  band_start, phase_count   Sec. 2.2 segments taken along rows
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "csc2d_oracle.c")
_SO = os.path.join(_HERE, "liboracle2d.so")
_lib = None

_i64 = ctypes.c_longlong
_dp = ctypes.POINTER(ctypes.c_double)
_fp = ctypes.POINTER(ctypes.c_float)
_ip = ctypes.POINTER(ctypes.c_int)
_lp = ctypes.POINTER(ctypes.c_longlong)
_c = ctypes.c_int


def build(force: bool = False) -> str:
    """Compile csc2d_oracle.c into liboracle2d.so (plain gcc, no FMA contraction)."""
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + ".%d.tmp" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-std=c11", "-fPIC", "-shared",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _SO)
    return _SO


def bind(path: str):
    lib = ctypes.CDLL(path)
    dims = [_c, _c, _c, _c]  # K, P, h, w
    lib.o2_norms.argtypes = [_fp, *dims, _dp]
    lib.o2_crosscorr.argtypes = [_fp, *dims, _dp]
    lib.o2_dtx.argtypes = [_fp, _fp, *dims, _i64, _i64, _dp]
    lib.o2_residual.argtypes = [_fp, _fp, _dp, *dims, _i64, _i64, _dp]
    lib.o2_objective.restype = ctypes.c_double
    lib.o2_objective.argtypes = [_fp, _fp, _dp, *dims, _i64, _i64, ctypes.c_double]
    lib.o2_beta_fresh.argtypes = [_fp, _fp, _dp, *dims, _i64, _i64, _dp]
    lib.o2_band_start.restype = _i64
    lib.o2_band_start.argtypes = [_i64, _c, _c]
    lib.o2_phase_count.restype = _c
    lib.o2_phase_count.argtypes = [_i64, _c, _c]
    lib.o2_greedy_cd.restype = _i64
    lib.o2_greedy_cd.argtypes = [_fp, _fp, *dims, _i64, _i64, ctypes.c_double, ctypes.c_double,
                                 _i64, _dp, _dp, _ip, _lp, _dp, _dp, _i64, _ip]
    lib.o2_locally_greedy_cd.restype = _i64
    lib.o2_locally_greedy_cd.argtypes = [_fp, _fp, *dims, _i64, _i64, ctypes.c_double,
                                         ctypes.c_double, _i64, _c, _c, ctypes.c_ulonglong, _c,
                                         _dp, _dp, _ip, _lp, _dp, _dp, _i64, _ip, _lp]
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


def _dims(D, X=None):
    K, P, h, w = (int(x) for x in D.shape)
    if X is None:
        return K, P, h, w
    return K, P, h, w, int(X.shape[1]), int(X.shape[2])


def norms(D) -> np.ndarray:
    D = _f32(D)
    K, P, h, w = _dims(D)
    out = np.empty(K, np.float64)
    _load().o2_norms(_p(D, _fp), K, P, h, w, _p(out, _dp))
    return out


def crosscorr(D) -> np.ndarray:
    """S[k, l, a, b] at lag (a - (h-1), b - (w-1)), shape [K, K, 2h-1, 2w-1]."""
    D = _f32(D)
    K, P, h, w = _dims(D)
    out = np.empty((K, K, 2 * h - 1, 2 * w - 1), np.float64)
    _load().o2_crosscorr(_p(D, _fp), K, P, h, w, _p(out, _dp))
    return out


def dtx(D, X) -> np.ndarray:
    D, X = _f32(D), _f32(X)
    K, P, h, w, H, W = _dims(D, X)
    out = np.empty((K, H - h + 1, W - w + 1), np.float64)
    _load().o2_dtx(_p(D, _fp), _p(X, _fp), K, P, h, w, H, W, _p(out, _dp))
    return out


def lambda_max(D, X) -> float:
    return float(np.max(np.abs(dtx(D, X))))


def residual(D, X, Z) -> np.ndarray:
    D, X, Z = _f32(D), _f32(X), _f64(Z)
    K, P, h, w, H, W = _dims(D, X)
    out = np.empty((P, H, W), np.float64)
    _load().o2_residual(_p(D, _fp), _p(X, _fp), _p(Z, _dp), K, P, h, w, H, W, _p(out, _dp))
    return out


def objective(D, X, Z, lam: float) -> float:
    D, X, Z = _f32(D), _f32(X), _f64(Z)
    K, P, h, w, H, W = _dims(D, X)
    return _load().o2_objective(_p(D, _fp), _p(X, _fp), _p(Z, _dp), K, P, h, w, H, W,
                                float(lam))


def beta_fresh(D, X, Z) -> np.ndarray:
    D, X, Z = _f32(D), _f32(X), _f64(Z)
    K, P, h, w, H, W = _dims(D, X)
    out = np.empty((K, H - h + 1, W - w + 1), np.float64)
    _load().o2_beta_fresh(_p(D, _fp), _p(X, _fp), _p(Z, _dp), K, P, h, w, H, W, _p(out, _dp))
    return out


def band_start(Hz: int, M: int, m: int) -> int:
    return int(_load().o2_band_start(Hz, M, m))


def phase_count(Hz: int, M: int, h: int) -> int:
    return int(_load().o2_phase_count(Hz, M, h))


def _trace(cap):
    return (np.zeros(cap, np.int32), np.zeros(cap, np.int64), np.zeros(cap, np.float64),
            np.zeros(cap, np.float64))


def _result(Z, beta, q, conv, tr, cap, Wz, sweeps=None):
    if q < 0:
        raise ValueError("invalid arguments or allocation failure")
    res = {"Z": Z, "beta": beta, "n_updates": int(q), "converged": bool(conv)}
    if sweeps is not None:
        res["sweeps"] = int(sweeps)
    if cap:
        n = min(int(q), cap)
        t = tr[1][:n]
        res["trace"] = {"k": tr[0][:n].copy(), "i": t // Wz, "j": t % Wz,
                        "z_old": tr[2][:n].copy(), "z_new": tr[3][:n].copy()}
    return res


def greedy_cd(D, X, lam: float, eps: float, max_updates: int = 10**9, trace: int = 0) -> dict:
    """Alg. 1 on the image.  Returns Z, beta (FP64), n_updates, converged (and trace)."""
    D, X = _f32(D), _f32(X)
    K, P, h, w, H, W = _dims(D, X)
    Z = np.zeros((K, H - h + 1, W - w + 1))
    beta = np.zeros_like(Z)
    tr = _trace(max(trace, 1))
    conv = ctypes.c_int(0)
    q = _load().o2_greedy_cd(_p(D, _fp), _p(X, _fp), K, P, h, w, H, W, float(lam), float(eps),
                             int(max_updates), _p(Z, _dp), _p(beta, _dp), _p(tr[0], _ip),
                             _p(tr[1], _lp), _p(tr[2], _dp), _p(tr[3], _dp), int(trace),
                             ctypes.byref(conv))
    return _result(Z, beta, q, conv.value, tr, trace, W - w + 1)


def locally_greedy_cd(D, X, lam: float, eps: float, M: int, mode: str = "phase", seed: int = 0,
                      updates_per_visit: int = 0, max_updates: int = 10**9,
                      trace: int = 0) -> dict:
    """Alg. 3 on M row bands: mode "random" (a band per step) or "phase"
    (the band phase schedule, ``updates_per_visit`` per visit, 0 = no limit)."""
    D, X = _f32(D), _f32(X)
    K, P, h, w, H, W = _dims(D, X)
    Z = np.zeros((K, H - h + 1, W - w + 1))
    beta = np.zeros_like(Z)
    tr = _trace(max(trace, 1))
    conv = ctypes.c_int(0)
    sweeps = ctypes.c_longlong(0)
    q = _load().o2_locally_greedy_cd(
        _p(D, _fp), _p(X, _fp), K, P, h, w, H, W, float(lam), float(eps), int(max_updates),
        int(M), 0 if mode == "random" else 1, int(seed), int(updates_per_visit), _p(Z, _dp),
        _p(beta, _dp), _p(tr[0], _ip), _p(tr[1], _lp), _p(tr[2], _dp), _p(tr[3], _dp), int(trace),
        ctypes.byref(conv), ctypes.byref(sweeps))
    return _result(Z, beta, q, conv.value, tr, trace, W - w + 1, sweeps.value)
