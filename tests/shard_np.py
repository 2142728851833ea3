"""A float64 numpy stand-in for one rank's csc_shard_* calls (include/csc_shard.h).

It runs the phase schedule of Alg. 3 on the rank's window in the beta form of
Sec. 2.1 (beta = D~*X - sum S Z with each coordinate's own term kept out),
with the same visit rules as the GPU phase kernel: a segment that needs a
visit repeats "argmax over the segment of |Z' - Z|, stop below tol or after u
updates, else Z <- Z' and Eq. beta_up on the window"; segments reached by a
window (or by a neighbour's change) need a visit again.  The halo columns
start at 0 and accumulate the changes the neighbours must apply.  This lets
the multi-process protocol in paper_1705_10087_gb300/shard.py run on CPU
ranks; it is test infrastructure and shares no code with the library.
"""
from __future__ import annotations

import numpy as np


def coupling(D):
    """C[k, l, d] = sum_p sum_tau D[k,p,tau] D[l,p,tau+d-(L-1)]: the change of
    beta_k[t] per unit change of Z_l[t0] is -C[k, l, t - t0 + L - 1]."""
    K, P, L = D.shape
    D = D.astype(np.float64)
    C = np.zeros((K, K, 2 * L - 1))
    for k in range(K):
        for l in range(K):
            for p in range(P):
                # correlate(a, v, 'full')[n] = sum_m a[m + n - (L-1)] v[m]
                C[k, l] += np.correlate(D[l, p], D[k, p], mode="full")
    return C


def dtx(D, X):
    K, P, L = D.shape
    Tz = X.shape[1] - L + 1
    out = np.zeros((K, Tz))
    for k in range(K):
        for p in range(P):
            out[k] += np.correlate(X[p].astype(np.float64), D[k, p].astype(np.float64), "valid")
    return out


def soft(u, lam):
    return np.sign(u) * np.maximum(np.abs(u) - lam, 0.0)


class NumpyShard:
    def __init__(self, D, Xw, plan, lam, u=24):
        self.D = D.astype(np.float64)
        self.K, self.P, self.L = D.shape
        self.X = Xw.astype(np.float64)
        self.plan = plan
        self.lam = float(lam)
        self.u = int(u)
        self.C = coupling(D)
        self.n = (self.D ** 2).sum(axis=(1, 2))
        self.beta0 = dtx(D, Xw)
        self.Tz = self.beta0.shape[1]
        self.hl, self.hr = int(plan["halo_left"]), int(plan["halo_right"])
        self.cc = int(plan["col_count"])
        self.beta = self.beta0.copy()
        self.beta[:, :self.hl] = 0.0
        self.beta[:, self.hl + self.cc:] = 0.0
        self.Z = np.zeros_like(self.beta0)
        Tzg, M = int(plan["Tz"]), int(plan["M"])
        s0, c0 = int(plan["seg_first"]), int(plan["col_first"])
        self.seg = [(m * Tzg // M - c0 + self.hl, (m + 1) * Tzg // M - c0 + self.hl)
                    for m in range(s0, s0 + int(plan["seg_count"]))]
        self.dirty = np.ones(len(self.seg), bool)
        self.total = 0
        self.sent = 0  # nonzero halo changes handed to the neighbours

    # -- csc_shard_phase
    def phase(self, p, tol):
        c, s0 = int(self.plan["phases"]), int(self.plan["seg_first"])
        L = self.L
        for i, (s, e) in enumerate(self.seg):
            if (s0 + i) % c != p or not self.dirty[i]:
                continue
            nupd, capped, tmin, tmax = 0, False, None, None
            while True:
                zp = soft(self.beta[:, s:e], self.lam) / self.n[:, None]
                dz = zp - self.Z[:, s:e]
                j = int(np.argmax(np.abs(dz)))  # lowest (k, t) among the largest
                k0, jj = divmod(j, e - s)
                if not abs(dz[k0, jj]) >= tol:
                    break
                if nupd >= self.u:
                    capped = True
                    break
                t0 = s + jj
                d = dz[k0, jj]
                self.Z[k0, t0] = zp[k0, jj]
                lo, hi = max(0, t0 - L + 1), min(self.Tz, t0 + L)
                own = self.beta[k0, t0]
                self.beta[:, lo:hi] -= self.C[:, k0, lo - t0 + L - 1:hi - t0 + L - 1] * d
                self.beta[k0, t0] = own  # Eq. beta_up skips the own coordinate
                nupd += 1
                tmin = t0 if tmin is None else min(tmin, t0)
                tmax = t0 if tmax is None else max(tmax, t0)
            self.dirty[i] = capped
            if nupd:
                for q, (a, b) in enumerate(self.seg):
                    if q != i and b > tmin - L + 1 and a <= tmax + L - 1:
                        self.dirty[q] = True
                self.total += nupd

    # -- halo and border exchange
    def halo_out(self, to_left, to_right):
        if self.hl:
            self.sent += int(np.count_nonzero(self.beta[:, :self.hl]))
            to_left[...] = _as(to_left, self.beta[:, :self.hl])
            self.beta[:, :self.hl] = 0.0
        if self.hr:
            a = self.hl + self.cc
            self.sent += int(np.count_nonzero(self.beta[:, a:a + self.hr]))
            to_right[...] = _as(to_right, self.beta[:, a:a + self.hr])
            self.beta[:, a:a + self.hr] = 0.0

    def halo_in(self, from_left, from_right):
        for blk, c0, w in ((from_left, self.hl, self.hl),
                           (from_right, self.hl + self.cc - self.hr, self.hr)):
            if not w:
                continue
            v = np.asarray(blk, np.float64)
            self.beta[:, c0:c0 + w] += v
            cols = c0 + np.nonzero(np.any(v != 0.0, axis=0))[0]
            for q, (a, b) in enumerate(self.seg):
                if np.any((cols >= a) & (cols < b)):
                    self.dirty[q] = True

    def z_out(self, to_left, to_right):
        if self.hl:
            to_left[...] = _as(to_left, self.Z[:, self.hl:2 * self.hl])
        if self.hr:
            a = self.hl + self.cc
            to_right[...] = _as(to_right, self.Z[:, a - self.hr:a])

    def z_in(self, from_left, from_right):
        if self.hl:
            self.Z[:, :self.hl] = np.asarray(from_left, np.float64)
        if self.hr:
            a = self.hl + self.cc
            self.Z[:, a:a + self.hr] = np.asarray(from_right, np.float64)

    def updates(self):
        return self.total

    # -- exact checks
    def _beta_owned(self):
        L, a, b = self.L, self.hl, self.hl + self.cc
        out = self.beta0[:, a:b].copy()
        for k in range(self.K):
            for l in range(self.K):
                # sum over t' of C[k, l, t - t' + L - 1] Z[l, t'] for t in [a, b)
                full = np.convolve(self.Z[l], self.C[k, l])  # index t + L - 1
                out[k] -= full[a + L - 1:b + L - 1]
        out += self.n[:, None] * self.Z[:, a:b]
        return out

    def resync(self, tol):
        a, b = self.hl, self.hl + self.cc
        beta = self._beta_owned()
        self.beta[:, a:b] = beta
        self.dirty[:] = True
        return float(np.abs(soft(beta, self.lam) / self.n[:, None] - self.Z[:, a:b]).max())

    def objective(self):
        L, a = self.L, self.hl
        R = self.X.copy()
        for k in range(self.K):
            for p in range(self.P):
                R[p] -= np.convolve(self.Z[k], self.D[k, p])
        end = a + self.cc + (L - 1 if self.hr == 0 else 0)
        return 0.5 * float((R[:, a:end] ** 2).sum()) + self.lam * float(
            np.abs(self.Z[:, a:a + self.cc]).sum())

    def get_z(self, out=None):
        z = self.Z[:, self.hl:self.hl + self.cc].copy()
        if out is not None:
            out[...] = _as(out, z)
            return out
        return z


def _as(like, v):
    """v converted for assignment into `like` (a numpy array or a torch tensor)."""
    if isinstance(like, np.ndarray):
        return v
    import torch
    return torch.from_numpy(np.ascontiguousarray(v)).to(like.dtype)


class LocalComm:
    """The communicator of a single rank: no neighbours."""

    def exchange(self, *a):
        pass

    def sum(self, v):
        return float(v)

    def max(self, v):
        return float(v)
