"""Pins of the 2-D variant's FP64 oracle (oracle/csc2d.py, images cut into row
bands) against what the mathematics fixes.

Comparisons are against scipy.signal routines (correlate, convolve2d), a
different algorithm (FISTA, exhaustive sign-pattern search), the already
pinned 1-D oracle (a one-row image is a 1-D signal), an invariance (the
transposed problem has the transposed optimum) or brute force over the band
schedule, never against the oracle itself.  Atoms have non-unit norms so that a
dropped ||D_k||^2 cannot hide.
"""
import numpy as np
import pytest

import oracle
from oracle import csc2d
from tests import npref

pytest.importorskip("scipy")

CAP = 60_000


def tiny2d(K=2, P=2, h=3, w=2, H=9, W=8, rho=0.1, sigma=0.05, seed=1):
    """Seeded 2-D problem: Gaussian atoms of norms 0.6..1.7, Bernoulli-Gaussian Z,
    X = sum_k Z_k * D_k + noise (float32)."""
    rng = np.random.default_rng(seed)
    D = rng.standard_normal((K, P, h, w))
    D /= np.sqrt((D ** 2).sum(axis=(1, 2, 3)))[:, None, None, None]
    D *= np.linspace(0.6, 1.7, K)[:, None, None, None]
    D = D.astype(np.float32)
    Hz, Wz = H - h + 1, W - w + 1
    Z = rng.standard_normal((K, Hz, Wz)) * (rng.random((K, Hz, Wz)) < rho)
    X = -npref.residual2d(D, np.zeros((P, H, W), np.float32), Z)
    X = (X + sigma * rng.standard_normal(X.shape)).astype(np.float32)
    return D, X


# ------------------------------------------------------------- definitions

def test_crosscorr_and_norms_match_scipy():
    D, _ = tiny2d(K=3, P=2, h=3, w=4)
    S = csc2d.crosscorr(D)
    np.testing.assert_allclose(S, npref.crosscorr2d(D), rtol=1e-13, atol=1e-14)
    # S_{k,l}[a, b] = S_{l,k}[-a, -b]; zero lag = ||D_k||^2
    np.testing.assert_allclose(S, np.transpose(S, (1, 0, 2, 3))[:, :, ::-1, ::-1], atol=1e-14)
    n = csc2d.norms(D)
    np.testing.assert_allclose(n, npref.norms2d(D), rtol=1e-14)
    np.testing.assert_allclose(S[np.arange(3), np.arange(3), 2, 3], n, rtol=1e-14)


def test_dtx_matches_scipy_valid_correlation():
    D, X = tiny2d(K=3, P=2, h=4, w=3, H=11, W=10)
    np.testing.assert_allclose(csc2d.dtx(D, X), npref.dtx2d(D, X), rtol=1e-12, atol=1e-13)


def test_objective_matches_scipy_convolution():
    D, X = tiny2d()
    rng = np.random.default_rng(3)
    Z = rng.standard_normal((2, 7, 7)) * (rng.random((2, 7, 7)) < 0.3)
    np.testing.assert_allclose(csc2d.residual(D, X, Z), npref.residual2d(D, X, Z), atol=1e-13)
    assert csc2d.objective(D, X, Z, 0.3) == pytest.approx(npref.objective2d(D, X, Z, 0.3),
                                                          rel=1e-13)


def test_beta_fresh_matches_definition():
    D, X = tiny2d()
    rng = np.random.default_rng(4)
    Z = rng.standard_normal((2, 7, 7)) * (rng.random((2, 7, 7)) < 0.3)
    np.testing.assert_allclose(csc2d.beta_fresh(D, X, Z), npref.beta_fresh2d(D, X, Z),
                               atol=1e-12)


def _beta_tracks_definition(run, D, X, qmax):
    for q in range(1, qmax):
        r = run(q)
        B = npref.beta_fresh2d(D, X, r["Z"])
        assert np.abs(r["beta"] - B).max() <= 1e-11 * max(1.0, np.abs(B).max()), q
        if r["n_updates"] < q:
            break


def test_greedy_beta_update_matches_fresh_residual():
    # Eq. beta_up in 2-D: after every update beta equals its definition
    D, X = tiny2d()
    lam = 0.05 * csc2d.lambda_max(D, X)
    _beta_tracks_definition(lambda q: csc2d.greedy_cd(D, X, lam, 1e-12, max_updates=q),
                            D, X, 40)


def test_band_schedule_border_updates_match_fresh_residual():
    # updates near a band border spill into the idle neighbouring bands
    D, X = tiny2d(h=2, H=14)
    lam = 0.05 * csc2d.lambda_max(D, X)
    _beta_tracks_definition(
        lambda q: csc2d.locally_greedy_cd(D, X, lam, 1e-12, M=6, mode="phase",
                                          updates_per_visit=2, max_updates=q), D, X, 40)


def test_each_update_lowers_E_by_prop_A1():
    # Prop. A.1 in 2-D: E(Z) - E(Z1) = n/2 (z^2 - u^2) - beta (z - u) + lam (|z| - |u|) >= 0,
    # and the new value is the 1-D minimiser Sh(beta, lam) / n
    D, X = tiny2d(seed=21)
    lam = 0.1 * csc2d.lambda_max(D, X)
    r = csc2d.greedy_cd(D, X, lam, 1e-10, trace=10_000, max_updates=CAP)
    tr = r["trace"]
    n = npref.norms2d(D)
    Z = np.zeros_like(r["Z"])
    E = npref.objective2d(D, X, Z, lam)
    for q in range(len(tr["k"])):
        k, i, j = int(tr["k"][q]), int(tr["i"][q]), int(tr["j"][q])
        z, u = tr["z_old"][q], tr["z_new"][q]
        assert Z[k, i, j] == z
        b = npref.beta_fresh2d(D, X, Z)[k, i, j]
        e = n[k] / 2 * (z * z - u * u) - b * (z - u) + lam * (abs(z) - abs(u))
        assert u == pytest.approx(npref.soft(b, lam) / n[k], abs=1e-12)
        Z[k, i, j] = u
        E1 = npref.objective2d(D, X, Z, lam)
        assert E - E1 == pytest.approx(e, abs=1e-10 * max(1.0, E))
        assert E1 <= E + 1e-12 * E
        E = E1
    np.testing.assert_array_equal(Z, r["Z"])


def test_lambda_above_lambda_max_gives_zero():
    D, X = tiny2d()
    lmax = float(np.abs(npref.dtx2d(D, X)).max())
    r = csc2d.greedy_cd(D, X, lmax * (1 + 1e-9), 1e-12, max_updates=CAP)
    assert r["converged"] and not r["Z"].any()
    r2 = csc2d.locally_greedy_cd(D, X, 2 * lmax, 1e-12, M=3, max_updates=CAP)
    assert r2["converged"] and r2["n_updates"] == 0


# ------------------------------------------------------ reductions, invariance

def test_one_row_image_is_the_1d_problem():
    # H = h = 1: the 2-D problem is the 1-D one with T = W, L = w, and Alg. 1
    # takes the same steps (same tie-break) in both oracles
    rng = np.random.default_rng(7)
    K, P, w, W = 3, 2, 5, 60
    D1 = (rng.standard_normal((K, P, w)) * np.linspace(0.6, 1.7, K)[:, None, None])
    D1 = D1.astype(np.float32)
    X1 = rng.standard_normal((P, W)).astype(np.float32)
    lam = 0.1 * oracle.lambda_max(D1, X1)
    g1 = oracle.greedy_cd(D1, X1, lam, 1e-12, trace=10_000, max_updates=CAP)
    g2 = csc2d.greedy_cd(D1[:, :, None, :], X1[:, None, :], lam, 1e-12, trace=10_000,
                         max_updates=CAP)
    assert g1["converged"] and g2["converged"]
    assert g1["n_updates"] == g2["n_updates"]
    np.testing.assert_array_equal(g1["trace"]["k"], g2["trace"]["k"])
    np.testing.assert_array_equal(g1["trace"]["t"], g2["trace"]["j"])
    assert not g2["trace"]["i"].any()
    np.testing.assert_allclose(g2["Z"][:, 0, :], g1["Z"], atol=1e-13)


def test_transposed_problem_has_transposed_optimum():
    D, X = tiny2d(h=3, w=2, H=9, W=8, seed=5)
    lam = 0.1 * csc2d.lambda_max(D, X)
    a = csc2d.greedy_cd(D, X, lam, 1e-13, max_updates=CAP)
    Dt, Xt = np.swapaxes(D, 2, 3).copy(), np.swapaxes(X, 1, 2).copy()
    b = csc2d.greedy_cd(Dt, Xt, lam, 1e-13, max_updates=CAP)
    assert a["converged"] and b["converged"]
    np.testing.assert_allclose(np.swapaxes(b["Z"], 1, 2), a["Z"], atol=1e-10)
    assert csc2d.objective(Dt, Xt, b["Z"], lam) == pytest.approx(
        csc2d.objective(D, X, a["Z"], lam), rel=1e-12)


# ------------------------------------------------------------- optimality

def test_matches_fista_optimum():
    D, X = tiny2d(K=2, P=1, h=2, w=3, H=6, W=7, rho=0.15, seed=9)
    A = npref.operator2d(D, 6, 7)
    x = X.astype(np.float64).ravel()
    lam = 0.1 * csc2d.lambda_max(D, X)
    zf = npref.fista(A, x, lam, tol=1e-12)
    assert npref.lasso_kkt(A, x, zf, lam) < 1e-11
    r = csc2d.greedy_cd(D, X, lam, 1e-14, max_updates=CAP)
    assert r["converged"]
    np.testing.assert_allclose(r["Z"].ravel(), zf, atol=1e-9)


def test_matches_exhaustive_lasso():
    # 2 atoms x 2 x 2 positions = 8 coordinates: every sign pattern is tried
    D, X = tiny2d(K=2, P=1, h=2, w=2, H=3, W=3, rho=0.4, sigma=0.3, seed=11)
    A = npref.operator2d(D, 3, 3)
    x = X.astype(np.float64).ravel()
    lam = 0.15 * csc2d.lambda_max(D, X)
    zb, Eb = npref.brute_force_lasso(A, x, lam)
    assert np.count_nonzero(zb) >= 2
    for r in (csc2d.greedy_cd(D, X, lam, 1e-14, max_updates=CAP),
              csc2d.locally_greedy_cd(D, X, lam, 1e-14, M=2, mode="phase", max_updates=CAP),
              csc2d.locally_greedy_cd(D, X, lam, 1e-14, M=2, mode="random", seed=3,
                                      max_updates=CAP)):
        assert r["converged"]
        np.testing.assert_allclose(r["Z"].ravel(), zb, atol=1e-10)
        assert csc2d.objective(D, X, r["Z"], lam) == pytest.approx(Eb, rel=1e-12)


def test_kkt_at_solution():
    # coordinate-wise optimality (Theorem A.1) on the flattened image
    D, X = tiny2d(K=3, P=2, h=3, w=3, H=12, W=11, seed=13)
    lam = 0.1 * csc2d.lambda_max(D, X)
    r = csc2d.greedy_cd(D, X, lam, 1e-12, max_updates=CAP)
    assert r["converged"]
    B = npref.beta_fresh2d(D, X, r["Z"])
    K = D.shape[0]
    rep = oracle.kkt(B.reshape(K, -1), r["Z"].reshape(K, -1), npref.norms2d(D), lam)
    assert rep["zero_excess"] <= 1e-9 and rep["max_delta_z"] <= 1e-11


# --------------------------------------------------- bands and their phases

def test_bands_partition_and_phases_are_disjoint():
    # co-active bands' update rows [s-h+1, e+h-1) never meet; one phase fewer would
    rng = np.random.default_rng(0)
    cases = [(int(rng.integers(1, 400)), 0, int(rng.integers(1, 30))) for _ in range(60)]
    cases += [(200, 10, 11), (7, 7, 3), (64, 4, 17)]
    for Hz, M, h in cases:
        if M == 0:
            M = int(rng.integers(1, Hz + 1))
        starts = [csc2d.band_start(Hz, M, m) for m in range(M + 1)]
        assert starts[0] == 0 and starts[-1] == Hz
        assert all(b > a for a, b in zip(starts, starts[1:]))
        c = csc2d.phase_count(Hz, M, h)
        assert 1 <= c <= M
        for m in range(M):
            for m2 in range(m + c, min(M, m + 4 * c), c):
                assert starts[m + 1] + h - 1 <= starts[m2] - (h - 1), (Hz, M, h, m, m2)
        if M > 1 and h > 1:
            assert (c - 2) * np.diff(starts).min() < 2 * h - 2 or c == M


def test_single_band_equals_greedy_trajectory():
    # M = 1: the band argmax is the global one (Alg. 3 -> Alg. 1)
    D, X = tiny2d(seed=17)
    lam = 0.1 * csc2d.lambda_max(D, X)
    g = csc2d.greedy_cd(D, X, lam, 1e-9, trace=10_000, max_updates=CAP)
    p = csc2d.locally_greedy_cd(D, X, lam, 1e-9, M=1, mode="phase", trace=10_000,
                                max_updates=CAP)
    # Alg. 1 applies its final sub-eps update before testing; the schedule tests first
    assert g["n_updates"] == p["n_updates"] + 1
    for key in ("k", "i", "j", "z_old", "z_new"):
        np.testing.assert_array_equal(g["trace"][key][:-1], p["trace"][key])


@pytest.mark.parametrize("M,u", [(2, 0), (3, 1), (5, 3), (1, 1)])
def test_band_schedules_reach_greedy_optimum(M, u):
    # Theorem conv_dcp along one axis: every band schedule reaches Z*
    D, X = tiny2d(K=2, P=2, h=2, w=3, H=14, W=9, seed=19)
    lam = 0.1 * csc2d.lambda_max(D, X)
    g = csc2d.greedy_cd(D, X, lam, 1e-13, max_updates=CAP)
    for mode in ("phase", "random"):
        r = csc2d.locally_greedy_cd(D, X, lam, 1e-13, M=M, mode=mode, seed=M,
                                    updates_per_visit=u, max_updates=CAP)
        assert r["converged"]
        np.testing.assert_allclose(r["Z"], g["Z"], atol=1e-10)
        if mode == "phase" and M == 1 and u == 1:
            # one update per sweep until a sweep applies none
            assert r["sweeps"] == r["n_updates"] + 1
