"""Seeded synthetic convolutional-sparse-coding problems.

This module only draws inputs: a dictionary D[K,P,L], a sparse activation
signal Z[K,T-L+1] and an observed signal X[P,T] built with the generative
model of Sec. 2.1 (Eq. model): X = sum_k Z_k * D_k + noise.  It contains none
of the solver's arithmetic (no correlation with D, no coordinate update, no
objective); the CPU oracle, the CUDA path, the tests and the benchmark all
take their inputs from here and compute everything else on their own.

Random numbers come from a counter-based generator (SplitMix64, Steele,
Lea & Flood, OOPSLA 2014) so that the same seed gives the same arrays on
every machine and numpy version: uniforms are exact functions of
(seed, stream, index); normals use the Box-Muller transform.

Recipe (Sec. 4, "Long convolutional Sparse Coding Signals"): every entry of D
is N(0,1) and each atom D_k (over its P x L entries) is rescaled to unit
l2 norm; Z_k[t] = Bernoulli(rho) * N(0, sigma_z^2); the noise is white
N(0, sigma^2).  Arrays are stored as float32.
"""
from __future__ import annotations

import dataclasses

import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def _mix64(x: np.ndarray) -> np.ndarray:
    """SplitMix64 output function (bijective 64-bit finaliser)."""
    x = x.copy()
    x ^= x >> np.uint64(30)
    x *= _M1
    x ^= x >> np.uint64(27)
    x *= _M2
    x ^= x >> np.uint64(31)
    return x


def _bits(seed: int, stream: int, n: int) -> np.ndarray:
    """n 64-bit words: SplitMix64 state seed' + (i+1)*golden, i = 0..n-1."""
    with np.errstate(over="ignore"):
        key = _mix64(np.array([(seed * 0x100000001B3 + stream * 0x632BE59BD9B4E019)
                               & 0xFFFFFFFFFFFFFFFF], dtype=np.uint64))[0]
        ctr = np.arange(1, n + 1, dtype=np.uint64)
        return _mix64(key + ctr * _GOLDEN)


def _bits_at(seed: int, stream: int, idx: np.ndarray) -> np.ndarray:
    """Words number idx (0-based) of the stream: _bits(seed, stream, n)[idx]."""
    with np.errstate(over="ignore"):
        key = _mix64(np.array([(seed * 0x100000001B3 + stream * 0x632BE59BD9B4E019)
                               & 0xFFFFFFFFFFFFFFFF], dtype=np.uint64))[0]
        ctr = np.asarray(idx, dtype=np.uint64) + np.uint64(1)
        return _mix64(key + ctr * _GOLDEN)


def _to_unit(b: np.ndarray) -> np.ndarray:
    return ((b >> np.uint64(11)).astype(np.float64) + 0.5) * (1.0 / 9007199254740992.0)


def uniform(seed: int, stream: int, n: int) -> np.ndarray:
    """n float64 uniforms in the open interval (0, 1)."""
    return _to_unit(_bits(seed, stream, n))


def uniform_at(seed: int, stream: int, idx: np.ndarray) -> np.ndarray:
    """uniform(seed, stream, n)[idx] without drawing the others."""
    return _to_unit(_bits_at(seed, stream, idx))


def _box_muller(u1: np.ndarray, u2: np.ndarray) -> np.ndarray:
    return np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * np.pi * u2)


def normal(seed: int, stream: int, n: int) -> np.ndarray:
    """n float64 standard normals (Box-Muller on two uniform streams)."""
    return _box_muller(uniform(seed, 2 * stream, n), uniform(seed, 2 * stream + 1, n))


def normal_at(seed: int, stream: int, idx: np.ndarray) -> np.ndarray:
    """normal(seed, stream, n)[idx] without drawing the others."""
    return _box_muller(uniform_at(seed, 2 * stream, idx), uniform_at(seed, 2 * stream + 1, idx))


def bernoulli_support(seed: int, stream: int, n: int, rho: float) -> np.ndarray:
    """Sorted indices of the successes of n Bernoulli(rho) trials, drawn as
    geometric gaps (the number of failures before each success is
    floor(log U / log(1 - rho)), U uniform): the same law as testing n
    uniforms against rho, at a cost proportional to the successes."""
    if rho <= 0.0 or n <= 0:
        return np.zeros(0, np.int64)
    if rho >= 1.0:
        return np.arange(n, dtype=np.int64)
    chunk = int(rho * n + 10.0 * np.sqrt(rho * n) + 16)
    gaps = []
    pos = -1
    j = 0
    while True:
        u = uniform_at(seed, stream, np.arange(j, j + chunk))
        g = np.floor(np.log(u) / np.log1p(-rho)).astype(np.int64) + 1
        idx = pos + np.cumsum(g)
        gaps.append(idx[idx < n])
        if idx[-1] >= n:
            break
        pos = int(idx[-1])
        j += chunk
    return np.concatenate(gaps)


@dataclasses.dataclass
class Problem:
    """One synthetic problem. D[K,P,L], Z_true[K,Tz], X[P,T], all float32."""
    D: np.ndarray
    Z_true: np.ndarray
    X: np.ndarray
    seed: int
    rho: float
    sigma: float

    @property
    def K(self) -> int:
        return self.D.shape[0]

    @property
    def P(self) -> int:
        return self.D.shape[1]

    @property
    def L(self) -> int:
        return self.D.shape[2]

    @property
    def T(self) -> int:
        return self.X.shape[1]

    @property
    def Tz(self) -> int:
        return self.T - self.L + 1


def make_dictionary(K: int, P: int, L: int, seed: int) -> np.ndarray:
    """K unit-norm Gaussian atoms of shape [P, L] (float32)."""
    D = normal(seed, 1, K * P * L).reshape(K, P, L)
    D /= np.sqrt((D * D).sum(axis=(1, 2), keepdims=True))
    return D.astype(np.float32)


def make_problem(K: int, P: int, L: int, T: int, rho: float, sigma: float,
                 seed: int, sigma_z: float = 1.0, D: np.ndarray | None = None,
                 support: str = "dense") -> Problem:
    """Draw D (unless given), a Bernoulli-Gaussian Z and X = sum_k Z_k*D_k + noise.

    support="dense" tests one uniform per coordinate against rho and takes the
    amplitude of coordinate i from normal number i; support="gaps" draws the
    same Bernoulli law as geometric gaps (bernoulli_support) and takes the
    amplitude of the j-th nonzero from normal number j (cheaper for long
    signals; a different sample).  The model sum is accumulated in float64
    from the float32 dictionary and the float32 activations, then rounded once
    to float32.
    """
    if T < L:
        raise ValueError("T must be >= L")
    if D is None:
        D = make_dictionary(K, P, L, seed)
    D = np.ascontiguousarray(D, dtype=np.float32)
    K, P, L = D.shape
    Tz = T - L + 1
    if support == "dense":
        nz = np.flatnonzero(uniform(seed, 3, K * Tz) < rho)
        amp = normal_at(seed, 4, nz)
    elif support == "gaps":
        nz = bernoulli_support(seed, 3, K * Tz, rho)
        amp = normal_at(seed, 4, np.arange(nz.size))
    else:
        raise ValueError(f"unknown support mode {support!r}")
    Z = np.zeros(K * Tz, np.float32)
    Z[nz] = (amp * sigma_z).astype(np.float32)
    Z = Z.reshape(K, Tz)

    X = np.zeros((P, T), dtype=np.float64)
    ks, ts = np.nonzero(Z)
    if ks.size:
        zv = Z[ks, ts].astype(np.float64)
        idx = (ts[:, None] + np.arange(L)[None, :]).ravel()
        for p in range(P):
            w = (zv[:, None] * D[ks, p, :].astype(np.float64)).ravel()
            X[p] += np.bincount(idx, weights=w, minlength=T)
    X += sigma * normal(seed, 5, P * T).reshape(P, T)
    return Problem(D=D, Z_true=Z, X=X.astype(np.float32), seed=seed, rho=rho, sigma=sigma)


@dataclasses.dataclass
class Problem2D:
    """One synthetic image problem (the 2-D variant, images cut into row bands).
    D[K,P,h,w], Z_true[K,H-h+1,W-w+1], X[P,H,W], all float32."""
    D: np.ndarray
    Z_true: np.ndarray
    X: np.ndarray
    seed: int
    rho: float
    sigma: float


def make_problem2d(K: int, P: int, h: int, w: int, H: int, W: int, rho: float, sigma: float,
                   seed: int) -> Problem2D:
    """The Sec. 4 recipe on images: K unit-norm Gaussian atoms [P, h, w], Z
    Bernoulli(rho)-Gaussian over every coordinate (one uniform each), X = sum_k
    Z_k * D_k (2-D, "valid" placement: activation (i, j) covers rows i..i+h-1
    and columns j..j+w-1) plus N(0, sigma^2) noise, summed in float64 and
    rounded once to float32.  The paper has no image workload; this one only
    carries its law over to two dimensions."""
    if H < h or W < w:
        raise ValueError("the image must be at least as large as the atoms")
    D = normal(seed, 11, K * P * h * w).reshape(K, P, h, w)
    D /= np.sqrt((D * D).sum(axis=(1, 2, 3), keepdims=True))
    D = D.astype(np.float32)
    Hz, Wz = H - h + 1, W - w + 1
    nz = np.flatnonzero(uniform(seed, 13, K * Hz * Wz) < rho)
    Z = np.zeros(K * Hz * Wz, np.float32)
    Z[nz] = normal_at(seed, 14, nz).astype(np.float32)
    Z = Z.reshape(K, Hz, Wz)
    X = np.zeros((P, H, W), np.float64)
    ks, iz, jz = np.nonzero(Z)
    for k, i, j in zip(ks, iz, jz):
        X[:, i:i + h, j:j + w] += float(Z[k, i, j]) * D[k].astype(np.float64)
    X += sigma * normal(seed, 15, P * H * W).reshape(P, H, W)
    return Problem2D(D=D, Z_true=Z, X=X.astype(np.float32), seed=seed, rho=rho, sigma=sigma)


# Workloads, named by what they are (shapes from the paper's Sec. 4 setting,
# scaled as stated).  "segments" lists the segment counts M exercised.
WORKLOADS = {
    # short single-channel signal: greedy CD and locally greedy CD, 10 segments
    "short_P1_K5_L16_T2000": dict(P=1, K=5, L=16, T=2000, rho=0.01, sigma=0.01,
                                  segments=(1, 10), tol=1e-6),
    # single long multichannel signal
    "long_P7_K25_L64_T200000": dict(P=7, K=25, L=64, T=200_000, rho=0.005, sigma=0.1,
                                    segments=(64, 256, 1024, 3072), tol=1e-6),
    # very long single-channel recording (about 1.4 h at 1 kHz)
    "verylong_P1_K25_L200_T5000000": dict(P=1, K=25, L=200, T=5_000_000, rho=0.002,
                                          sigma=0.1, segments=(12_500,), tol=1e-6),
}


# Batches: n signals with lengths uniform in [T_min, T_max], one shared dictionary.
BATCH_WORKLOADS = {
    # 512 multichannel signals of uneven length against one dictionary
    "batch_P7_K25_L64_n512_T10000_500000": dict(P=7, K=25, L=64, n=512, T_min=10_000,
                                                T_max=500_000, rho=0.005, sigma=0.1, tol=1e-6),
}


def batch_lengths(n: int, T_min: int, T_max: int, seed: int) -> np.ndarray:
    """n lengths uniform on the integers [T_min, T_max]."""
    u = uniform(seed, 6, n)
    return np.minimum(T_min + np.floor(u * (T_max - T_min + 1)), T_max).astype(np.int64)


def batch_signal(name: str, seed: int, i: int, T: int) -> Problem:
    """Signal i of a batch workload: seed (seed << 20) + 1 + i, the dictionary
    of `seed`, the Bernoulli support drawn as geometric gaps."""
    w = BATCH_WORKLOADS[name]
    D = make_dictionary(w["K"], w["P"], w["L"], seed)
    return make_problem(K=w["K"], P=w["P"], L=w["L"], T=int(T), rho=w["rho"], sigma=w["sigma"],
                        seed=(seed << 20) + 1 + i, D=D, support="gaps")


def _batch_signal_args(args):
    return batch_signal(*args)


def make_batch(name: str, seed: int = 0, n: int | None = None, T_max: int | None = None,
               workers: int = 0) -> list:
    """Problems of a named batch workload, sharing the dictionary of `seed`.

    n and T_max may be reduced for smaller cases (lengths are then drawn for
    the reduced range).  workers > 1 draws the signals in that many spawned
    processes (same arrays as workers = 0)."""
    w = BATCH_WORKLOADS[name]
    n = n if n is not None else w["n"]
    T_max = T_max if T_max is not None else w["T_max"]
    T_min = min(w["T_min"], T_max)
    T = batch_lengths(n, T_min, T_max, seed)
    args = [(name, seed, i, int(T[i])) for i in range(n)]
    if workers > 1 and n > 1:
        import multiprocessing as mp
        with mp.get_context("spawn").Pool(min(workers, n)) as pool:
            return pool.map(_batch_signal_args, args, chunksize=max(1, n // (4 * workers)))
    return [batch_signal(*a) for a in args]


# Request streams: Poisson arrivals of signals with log-uniform lengths, each
# for one of several resident dictionaries (K, L, P) drawn uniformly.
SERVE_WORKLOADS = {
    "serve_4dict_poisson200_T5000_2000000": dict(
        rate=200.0, T_min=5_000, T_max=2_000_000, rho=0.005, sigma=0.1, lambda_frac=0.1,
        tol=1e-3, budget_bytes=40 << 30,
        dicts=((25, 64, 1), (25, 128, 7), (64, 64, 7), (64, 128, 1))),  # (K, L, P)
}


def serve_sources(name: str, seed: int = 0, T_source: int | None = None, workers: int = 0):
    """One long synthetic recording per dictionary of a request stream: a list
    of Problems (dictionary of seed (seed << 8) + j, T_source samples, default
    the longest request).  Requests are windows of these recordings."""
    w = SERVE_WORKLOADS[name]
    T = int(T_source if T_source is not None else w["T_max"])
    args = [(K, P, L, T, w["rho"], w["sigma"], (seed << 8) + j)
            for j, (K, L, P) in enumerate(w["dicts"])]
    if workers > 1:
        import multiprocessing as mp
        with mp.get_context("spawn").Pool(min(workers, len(args))) as pool:
            return pool.map(_serve_source_args, args)
    return [_serve_source_args(a) for a in args]


def _serve_source_args(a):
    K, P, L, T, rho, sigma, s = a
    return make_problem(K=K, P=P, L=L, T=T, rho=rho, sigma=sigma, seed=s, support="gaps")


def serve_schedule(name: str, n: int, seed: int = 0, T_max: int | None = None) -> dict:
    """The first n requests of a stream: arrival times (s, Poisson process at
    the stream's rate), dictionary index (uniform), length (log-uniform on
    [T_min, T_max]) and window offset into the dictionary's recording (uniform)."""
    w = SERVE_WORKLOADS[name]
    T_max = int(T_max if T_max is not None else w["T_max"])
    T_min = min(int(w["T_min"]), T_max)
    gaps = -np.log(uniform(seed, 20, n)) / w["rate"]
    dict_idx = np.minimum((uniform(seed, 21, n) * len(w["dicts"])).astype(np.int64),
                          len(w["dicts"]) - 1)
    u = uniform(seed, 22, n)
    T = np.floor(np.exp(np.log(T_min) + u * (np.log(T_max) - np.log(T_min)))).astype(np.int64)
    T = np.clip(T, T_min, T_max)
    frac = uniform(seed, 23, n)
    return {"arrival": np.cumsum(gaps), "dict": dict_idx, "T": T, "offset_frac": frac}


# Images for the 2-D variant (the paper has no image workload: the Sec. 4 law
# on one gray image, atoms of 8 x 8 pixels).
IMAGE_WORKLOADS = {
    "image_P1_K8_h8_w8_512x512": dict(K=8, P=1, h=8, w=8, H=512, W=512, rho=0.005, sigma=0.1,
                                      tol=1e-6),
}


def make_image_workload(name: str, seed: int = 0):
    w = IMAGE_WORKLOADS[name]
    return make_problem2d(K=w["K"], P=w["P"], h=w["h"], w=w["w"], H=w["H"], W=w["W"],
                          rho=w["rho"], sigma=w["sigma"], seed=seed)


def make_workload(name: str, seed: int = 0, T: int | None = None) -> Problem:
    """Problem for a named workload; T may be overridden for reduced-size cases."""
    w = WORKLOADS[name]
    return make_problem(K=w["K"], P=w["P"], L=w["L"], T=T if T is not None else w["T"],
                        rho=w["rho"], sigma=w["sigma"], seed=seed)
