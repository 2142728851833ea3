"""Multi-core CPU baseline (benchmark only): the oracle's FP64 segment phase
schedule with OpenMP over the segments of a phase (csc_baseline_omp.c).

Used by bench.py's CPU legs and by the test that checks it reproduces the
single-threaded oracle exactly.  Shares no code with the CUDA path.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "csc_baseline_omp.c")
_SO = os.path.join(_HERE, "libbaseline_omp.so")
_lib = None


def build(force: bool = False) -> str:
    """gcc with OpenMP (falls back to a single-threaded build without it)."""
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + ".%d.tmp" % os.getpid()
        base = ["gcc", "-O2", "-ffp-contract=off", "-std=c11", "-fPIC", "-shared", "-o", tmp,
                _SRC, "-lm"]
        if subprocess.call(base[:1] + ["-fopenmp"] + base[1:], stderr=subprocess.DEVNULL) != 0:
            subprocess.check_call(base)
        os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        dp = ctypes.POINTER(ctypes.c_double)
        fp = ctypes.POINTER(ctypes.c_float)
        lib.omp_phase_cd.restype = ctypes.c_longlong
        lib.omp_phase_cd.argtypes = [fp, fp, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                     ctypes.c_longlong, ctypes.c_double, ctypes.c_double,
                                     ctypes.c_int, ctypes.c_int, ctypes.c_int, dp, dp,
                                     ctypes.POINTER(ctypes.c_int),
                                     ctypes.POINTER(ctypes.c_longlong)]
        lib.omp_threads_used.restype = ctypes.c_int
        _lib = lib
    return _lib


def phase_cd(D, X, lam: float, eps: float, M: int, updates_per_visit: int = 0,
             threads: int = 0) -> dict:
    """Z, beta, updates, sweeps, converged and the threads used."""
    D = np.ascontiguousarray(D, np.float32)
    X = np.ascontiguousarray(X, np.float32)
    K, P, L = D.shape
    T = X.shape[1]
    Tz = T - L + 1
    Z = np.zeros((K, Tz))
    beta = np.zeros((K, Tz))
    conv = ctypes.c_int(0)
    sweeps = ctypes.c_longlong(0)
    lib = _load()
    q = lib.omp_phase_cd(D.ctypes.data_as(ctypes.POINTER(ctypes.c_float)),
                         X.ctypes.data_as(ctypes.POINTER(ctypes.c_float)), K, P, L, T,
                         float(lam), float(eps), int(M), int(updates_per_visit), int(threads),
                         Z.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                         beta.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                         ctypes.byref(conv), ctypes.byref(sweeps))
    if q < 0:
        raise ValueError("omp_phase_cd: bad arguments")
    return {"Z": Z, "beta": beta, "n_updates": int(q), "sweeps": int(sweeps.value),
            "converged": bool(conv.value), "threads": int(lib.omp_threads_used())}
