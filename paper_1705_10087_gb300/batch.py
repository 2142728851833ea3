"""Layout helpers for batches of signals (csc_init_batch).

A batch of n signals X_i [P, T_i] is passed to the library concatenated in
time, X [P, sum T_i]; its activations come back the same way, Z [K, sum T_i -
L + 1], where signal i owns the columns [a_i, a_i + T_i - L + 1) with
a_i = T_0 + ... + T_{i-1}.  The L - 1 columns after each signal's last valid
column straddle two signals and hold 0.  These helpers only move data.
"""
from __future__ import annotations

import numpy as np


def offsets(T) -> np.ndarray:
    """Sample offsets a[0..n] of the concatenation (a[0] = 0, a[n] = sum T)."""
    T = np.asarray(T, dtype=np.int64).reshape(-1)
    return np.concatenate([[0], np.cumsum(T)]).astype(np.int64)


def pack(Xs) -> tuple[np.ndarray, np.ndarray]:
    """List of [P, T_i] arrays -> (X [P, sum T_i] float32, T [n] int64)."""
    if not Xs:
        raise ValueError("a batch needs at least one signal")
    P = Xs[0].shape[0]
    if any(x.ndim != 2 or x.shape[0] != P for x in Xs):
        raise ValueError("every signal must be [P, T_i] with the same P")
    T = np.array([x.shape[1] for x in Xs], dtype=np.int64)
    X = np.ascontiguousarray(np.concatenate(Xs, axis=1), dtype=np.float32)
    return X, T


def pack_Z(Zs, L: int) -> np.ndarray:
    """List of [K, T_i - L + 1] activations -> the concatenated [K, sum T_i - L + 1]
    (straddling columns 0), e.g. for a warm start."""
    K = Zs[0].shape[0]
    T = np.array([z.shape[1] + L - 1 for z in Zs], dtype=np.int64)
    a = offsets(T)
    Z = np.zeros((K, int(a[-1]) - L + 1), np.float32)
    for i, z in enumerate(Zs):
        Z[:, a[i]:a[i] + z.shape[1]] = z
    return Z


def unpack_Z(Z, T, L: int) -> list:
    """Concatenated Z [K, sum T - L + 1] -> per-signal views [K, T_i - L + 1]."""
    a = offsets(T)
    return [Z[:, a[i]:a[i + 1] - L + 1] for i in range(len(a) - 1)]


def straddle_mask(T, L: int) -> np.ndarray:
    """Boolean [sum T - L + 1]: True on the columns that belong to no signal."""
    a = offsets(T)
    m = np.ones(int(a[-1]) - L + 1, dtype=bool)
    for i in range(len(a) - 1):
        m[a[i]:a[i + 1] - L + 1] = False
    return m
