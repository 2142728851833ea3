"""Independent numpy computations used to pin the FP64 oracle.

Everything here is built from library primitives (np.correlate, np.convolve,
np.fft, np.linalg) or from a different algorithm (FISTA, exhaustive search
over sign patterns), never from the oracle's own loops, so that agreement
with the oracle is evidence and not a tautology.
"""
from __future__ import annotations

import itertools

import numpy as np


def crosscorr(D):
    """S[k,l,s] = sum_p correlate(D_l[p], D_k[p], 'full')[s]."""
    K, P, L = D.shape
    D = D.astype(np.float64)
    S = np.zeros((K, K, 2 * L - 1))
    for k in range(K):
        for l in range(K):
            for p in range(P):
                S[k, l] += np.correlate(D[l, p], D[k, p], mode="full")
    return S


def dtx_fft(D, X):
    """beta0[k,t] = sum_p sum_tau D[k,p,tau] X[p,t+tau] through real FFTs."""
    K, P, L = D.shape
    T = X.shape[1]
    Tz = T - L + 1
    n = 1 << int(np.ceil(np.log2(T + L)))
    FX = np.fft.rfft(X.astype(np.float64), n, axis=1)
    FD = np.fft.rfft(D.astype(np.float64), n, axis=2)
    out = np.zeros((K, Tz))
    for k in range(K):
        out[k] = np.fft.irfft((FX * np.conj(FD[k])).sum(axis=0), n)[:Tz]
    return out


def residual(D, X, Z):
    """X - sum_k Z_k * D_k with np.convolve (full convolution has length T)."""
    K, P, L = D.shape
    R = X.astype(np.float64).copy()
    for k in range(K):
        for p in range(P):
            R[p] -= np.convolve(Z[k].astype(np.float64), D[k, p].astype(np.float64))
    return R


def objective(D, X, Z, lam):
    R = residual(D, X, Z)
    return 0.5 * float((R * R).sum()) + lam * float(np.abs(Z).sum())


def norms(D):
    return (D.astype(np.float64) ** 2).sum(axis=(1, 2))


def beta_fresh(D, X, Z):
    """Correlation of each atom with the residual, own coordinate put back."""
    K, P, L = D.shape
    R = residual(D, X, Z)
    n = norms(D)
    B = np.zeros(Z.shape)
    for k in range(K):
        for p in range(P):
            B[k] += np.correlate(R[p], D[k, p].astype(np.float64), mode="valid")
        B[k] += n[k] * Z[k]
    return B


def operator(D, T):
    """Dense matrix A of Z -> vec(sum_k Z_k * D_k), shape (P*T, K*Tz)."""
    K, P, L = D.shape
    Tz = T - L + 1
    A = np.zeros((P * T, K * Tz))
    for k in range(K):
        for t in range(Tz):
            e = np.zeros(Tz)
            e[t] = 1.0
            A[:, k * Tz + t] = np.concatenate(
                [np.convolve(e, D[k, p].astype(np.float64)) for p in range(P)])
    return A


def soft(u, lam):
    return np.sign(u) * np.maximum(np.abs(u) - lam, 0.0)


def lasso_kkt(A, x, z, lam):
    g = A.T @ (x - A @ z)
    nz = z != 0
    v_nz = np.abs(g[nz] - lam * np.sign(z[nz])).max(initial=0.0)
    v_z = np.maximum(np.abs(g[~nz]) - lam, 0.0).max(initial=0.0)
    return max(v_nz, v_z)


def fista(A, x, lam, tol=1e-12, max_iter=200_000):
    """FISTA (Beck & Teboulle 2009) with gradient-based adaptive restart
    (O'Donoghue & Candes 2015); step 1/||A||_2^2."""
    Lip = np.linalg.norm(A, 2) ** 2
    z = np.zeros(A.shape[1])
    y = z.copy()
    tk = 1.0
    for it in range(max_iter):
        g = A.T @ (A @ y - x)
        z_new = soft(y - g / Lip, lam / Lip)
        if np.dot(y - z_new, z_new - z) > 0:   # restart
            tk = 1.0
            y = z_new.copy()
        else:
            t_next = 0.5 * (1 + np.sqrt(1 + 4 * tk * tk))
            y = z_new + ((tk - 1) / t_next) * (z_new - z)
            tk = t_next
        z = z_new
        if it % 50 == 0 and lasso_kkt(A, x, z, lam) < tol:
            break
    return z


def brute_force_lasso(A, x, lam):
    """Exact LASSO minimiser by trying every sign pattern s in {-1,0,1}^n:
    on the support the optimum solves A_S^T A_S z = A_S^T x - lam s_S, and it
    is admissible when sign(z_S) == s_S.  Returns (z, E)."""
    n = A.shape[1]
    best = (np.zeros(n), 0.5 * float(x @ x))
    for s in itertools.product((-1, 0, 1), repeat=n):
        s = np.array(s, dtype=np.float64)
        S = np.nonzero(s)[0]
        if S.size == 0:
            continue
        As = A[:, S]
        G = As.T @ As
        zs = np.linalg.solve(G, As.T @ x - lam * s[S])
        if np.any(np.sign(zs) != s[S]):
            continue
        z = np.zeros(n)
        z[S] = zs
        r = x - A @ z
        E = 0.5 * float(r @ r) + lam * float(np.abs(z).sum())
        if E < best[1]:
            best = (z, E)
    return best


# ------------------------------------------------- 2-D (scipy.signal routines)

def _signal():
    import scipy.signal
    return scipy.signal


def crosscorr2d(D):
    """S[k,l,a,b] = sum_p correlate(D_l[p], D_k[p], 'full')[a, b] (scipy.signal)."""
    sig = _signal()
    K, P, h, w = D.shape
    D = D.astype(np.float64)
    S = np.zeros((K, K, 2 * h - 1, 2 * w - 1))
    for k in range(K):
        for l in range(K):
            for p in range(P):
                S[k, l] += sig.correlate(D[l, p], D[k, p], mode="full", method="direct")
    return S


def dtx2d(D, X):
    """beta0[k,i,j] = sum_p sum_{u,v} D[k,p,u,v] X[p,i+u,j+v] (scipy 'valid' correlation)."""
    sig = _signal()
    K, P, h, w = D.shape
    out = None
    for k in range(K):
        acc = sum(sig.correlate(X[p].astype(np.float64), D[k, p].astype(np.float64),
                                mode="valid", method="direct") for p in range(P))
        if out is None:
            out = np.zeros((K,) + acc.shape)
        out[k] = acc
    return out


def residual2d(D, X, Z):
    """X - sum_k Z_k * D_k with scipy's full 2-D convolution (size H x W)."""
    sig = _signal()
    K, P, h, w = D.shape
    R = X.astype(np.float64).copy()
    for k in range(K):
        for p in range(P):
            R[p] -= sig.convolve2d(Z[k].astype(np.float64), D[k, p].astype(np.float64),
                                   mode="full")
    return R


def objective2d(D, X, Z, lam):
    R = residual2d(D, X, Z)
    return 0.5 * float((R * R).sum()) + lam * float(np.abs(Z).sum())


def norms2d(D):
    return (D.astype(np.float64) ** 2).sum(axis=(1, 2, 3))


def beta_fresh2d(D, X, Z):
    n = norms2d(D)
    return dtx2d(D, residual2d(D, X, Z)) + n[:, None, None] * Z


def operator2d(D, H, W):
    """Dense matrix of Z -> vec(sum_k Z_k * D_k), shape (P*H*W, K*Hz*Wz)."""
    sig = _signal()
    K, P, h, w = D.shape
    Hz, Wz = H - h + 1, W - w + 1
    A = np.zeros((P * H * W, K * Hz * Wz))
    for k in range(K):
        for i in range(Hz):
            for j in range(Wz):
                e = np.zeros((Hz, Wz))
                e[i, j] = 1.0
                A[:, (k * Hz + i) * Wz + j] = np.concatenate(
                    [sig.convolve2d(e, D[k, p].astype(np.float64), mode="full").ravel()
                     for p in range(P)])
    return A
