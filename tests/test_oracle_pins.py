"""Pins of the FP64 oracle against what the paper and mathematics fix.

Each test names the passage it checks.  The comparisons are against numpy
library routines, a different algorithm (FISTA, exhaustive search) or closed
forms, never against the oracle itself.  Tiny problems use atoms of non-unit
norm so that a dropped ||D_k||^2 cannot hide.
"""
import numpy as np
import pytest

import oracle
from paper_1705_10087_gb300 import synth
from tests import npref

# every solve in these pins is bounded, so that a broken oracle fails instead of looping
CAP = 50_000


def tiny(K=3, P=2, L=5, T=40, rho=0.08, sigma=0.05, seed=1, scale=True):
    pb = synth.make_problem(K=K, P=P, L=L, T=T, rho=rho, sigma=sigma, seed=seed)
    D = pb.D
    if scale:
        D = (D * np.linspace(0.6, 1.7, K, dtype=np.float32)[:, None, None]).astype(np.float32)
        pb = synth.make_problem(K=K, P=P, L=L, T=T, rho=rho, sigma=sigma, seed=seed, D=D)
    return pb


# ---------------------------------------------------------------- Sec. 2.1

@pytest.mark.parametrize("u,lam,want", [(3.0, 1.0, 2.0), (-3.0, 1.0, -2.0), (0.5, 1.0, 0.0),
                                        (-0.5, 1.0, 0.0), (1.0, 1.0, 0.0), (-1.0, 1.0, 0.0),
                                        (2.5, 0.0, 2.5)])
def test_soft_threshold_textbook(u, lam, want):
    # Sh(u, lam) = sign(u) max(|u| - lam, 0) (Sec. 2.1); |u| == lam gives 0.
    assert oracle.soft_threshold(u, lam) == want


def test_norms_and_crosscorr_match_numpy_correlate():
    pb = tiny(K=4, P=3, L=7)
    S = oracle.crosscorr(pb.D)
    np.testing.assert_allclose(S, npref.crosscorr(pb.D), rtol=0, atol=1e-13)
    n = oracle.norms(pb.D)
    np.testing.assert_allclose(n, npref.norms(pb.D), rtol=1e-14)
    L = pb.L
    # zero lag is the squared norm; S_{k,l}[t] = S_{l,k}[-t]
    np.testing.assert_allclose(np.diagonal(S[:, :, L - 1]), n, rtol=1e-14)
    np.testing.assert_allclose(S, np.transpose(S, (1, 0, 2))[:, :, ::-1], rtol=0, atol=1e-14)


def test_dtx_matches_fft_correlation():
    pb = synth.make_problem(K=5, P=3, L=16, T=700, rho=0.02, sigma=0.1, seed=3)
    b = oracle.dtx(pb.D, pb.X)
    ref = npref.dtx_fft(pb.D, pb.X)
    assert np.abs(b - ref).max() <= 1e-12 * max(1.0, np.abs(ref).max())


def test_objective_matches_numpy_convolution():
    pb = tiny()
    Z = np.random.default_rng(0).standard_normal((pb.K, pb.Tz)) * (
        np.random.default_rng(1).random((pb.K, pb.Tz)) < 0.2)
    lam = 0.3
    assert oracle.objective(pb.D, pb.X, Z, lam) == pytest.approx(
        npref.objective(pb.D, pb.X, Z, lam), rel=1e-13)
    np.testing.assert_allclose(oracle.residual(pb.D, pb.X, Z), npref.residual(pb.D, pb.X, Z),
                               rtol=0, atol=1e-13)


def test_beta_fresh_matches_definition():
    # beta_k[t]: correlation of D_k with the residual that excludes Z_k[t] (Sec. 2.1)
    pb = tiny()
    Z = np.random.default_rng(2).standard_normal((pb.K, pb.Tz)) * (
        np.random.default_rng(3).random((pb.K, pb.Tz)) < 0.3)
    B = oracle.beta_fresh(pb.D, pb.X, Z)
    np.testing.assert_allclose(B, npref.beta_fresh(pb.D, pb.X, Z), rtol=0, atol=1e-12)
    # brute force at one coordinate: put Z_k[t] to zero, correlate
    k, t = 1, 7
    Z0 = Z.copy()
    Z0[k, t] = 0.0
    R0 = npref.residual(pb.D, pb.X, Z0)
    direct = sum(float(pb.D[k, p].astype(np.float64) @ R0[p, t:t + pb.L]) for p in range(pb.P))
    assert B[k, t] == pytest.approx(direct, abs=1e-12)


# --------------------------------------------------- Alg. 1 / Eq. beta_up

def _check_beta_tracks_definition(run, pb, lam, n_max):
    """beta kept by Eq. beta_up equals the definition after every update."""
    for q in range(1, n_max + 1):
        r = run(q)
        fresh = npref.beta_fresh(pb.D, pb.X, r["Z"])
        err = np.abs(r["beta"] - fresh).max()
        assert err <= 1e-12, (q, err)
        if r["converged"]:
            break


def test_greedy_beta_update_matches_fresh_residual():
    pb = tiny()
    lam = 0.1 * oracle.lambda_max(pb.D, pb.X)
    _check_beta_tracks_definition(lambda q: oracle.greedy_cd(pb.D, pb.X, lam, 1e-12, max_updates=q),
                                  pb, lam, 60)


def test_phase_schedule_border_updates_match_fresh_residual():
    # updates near a segment border spill into the idle neighbour (Sec. 2.2, Fig. DCP)
    pb = tiny(T=60)
    lam = 0.05 * oracle.lambda_max(pb.D, pb.X)
    _check_beta_tracks_definition(
        lambda q: oracle.locally_greedy_cd(pb.D, pb.X, lam, 1e-12, M=6, mode="phase",
                                           updates_per_visit=2, max_updates=q), pb, lam, 60)


def test_each_update_lowers_E_by_prop_A1():
    # E(Z) - E(Z1) = n/2 (z^2 - u^2) - beta (z - u) + lam (|z| - |u|) >= 0 (Prop. A.1)
    pb = tiny()
    lam = 0.1 * oracle.lambda_max(pb.D, pb.X)
    r = oracle.greedy_cd(pb.D, pb.X, lam, 1e-10, trace=100_000, max_updates=CAP)
    tr = r["trace"]
    n = npref.norms(pb.D)
    Z = np.zeros((pb.K, pb.Tz))
    E = npref.objective(pb.D, pb.X, Z, lam)
    for i in range(len(tr["k"])):
        k, t, z, u = int(tr["k"][i]), int(tr["t"][i]), tr["z_old"][i], tr["z_new"][i]
        assert Z[k, t] == z
        b = npref.beta_fresh(pb.D, pb.X, Z)[k, t]
        e = n[k] / 2 * (z * z - u * u) - b * (z - u) + lam * (abs(z) - abs(u))
        Z[k, t] = u
        E1 = npref.objective(pb.D, pb.X, Z, lam)
        assert E - E1 == pytest.approx(e, abs=1e-10 * max(1.0, E))
        assert E1 <= E + 1e-12 * E
        # the chosen value is the 1-D minimiser of Eq. pb_coord
        assert u == pytest.approx(npref.soft(b, lam) / n[k], abs=1e-12)
        E = E1
    np.testing.assert_array_equal(Z, r["Z"])


def test_lambda_above_lambda_max_gives_zero():
    # with Z = 0 every Z' = Sh(D~*X, lam)/n vanishes once lam >= max|D~*X| (Alg. 1)
    pb = tiny()
    lmax = float(np.abs(npref.dtx_fft(pb.D, pb.X)).max())
    for lam in (lmax * (1 + 1e-9), 2 * lmax):
        r = oracle.greedy_cd(pb.D, pb.X, lam, 1e-12, max_updates=CAP)
        assert not r["Z"].any()
        assert r["converged"]
        r2 = oracle.locally_greedy_cd(pb.D, pb.X, lam, 1e-12, M=4, mode="phase", max_updates=CAP)
        assert not r2["Z"].any() and r2["n_updates"] == 0


def test_first_update_just_below_lambda_max():
    pb = tiny()
    b0 = npref.dtx_fft(pb.D, pb.X)
    n = npref.norms(pb.D)
    # largest |Delta Z| at Z=0 is max |Sh(b0,lam)|/n_k
    lam = 0.9 * float(np.abs(b0).max())
    r = oracle.greedy_cd(pb.D, pb.X, lam, 1e-12, max_updates=1, trace=1)
    cand = np.abs(npref.soft(b0, lam)) / n[:, None]
    k, t = np.unravel_index(np.argmax(cand), cand.shape)
    assert (r["trace"]["k"][0], r["trace"]["t"][0]) == (k, t)
    assert r["trace"]["z_new"][0] == pytest.approx(npref.soft(b0[k, t], lam) / n[k], rel=1e-13)


def test_closed_form_for_non_overlapping_atoms():
    # T = L (one time position) and atoms on disjoint channels: the Gram matrix
    # is diagonal, so Z_k = Sh(D_k^T X, lam) / ||D_k||^2 exactly (Eq. pb_coord).
    K, L = 4, 9
    rng = np.random.default_rng(5)
    D = np.zeros((K, K, L), np.float32)
    for k in range(K):
        D[k, k] = rng.standard_normal(L) * (0.5 + k)
    X = rng.standard_normal((K, L)).astype(np.float32) * 3
    lam = 0.7
    r = oracle.greedy_cd(D, X, lam, 1e-14, max_updates=CAP)
    assert r["converged"]
    want = np.array([npref.soft(float(D[k, k].astype(np.float64) @ X[k]), lam) /
                     float((D[k, k].astype(np.float64) ** 2).sum()) for k in range(K)])
    np.testing.assert_allclose(r["Z"][:, 0], want, rtol=1e-13, atol=1e-15)
    assert np.count_nonzero(want) >= 2


# ------------------------------------------------------------ optimality

def test_matches_fista_optimum():
    pb = tiny(K=2, P=3, L=6, T=40, rho=0.1, sigma=0.05, seed=7)
    A = npref.operator(pb.D, pb.T)
    x = pb.X.astype(np.float64).ravel()
    lam = 0.1 * oracle.lambda_max(pb.D, pb.X)
    zf = npref.fista(A, x, lam, tol=1e-12)
    assert npref.lasso_kkt(A, x, zf, lam) < 1e-11
    r = oracle.greedy_cd(pb.D, pb.X, lam, 1e-14, max_updates=CAP)
    assert r["converged"]
    np.testing.assert_allclose(r["Z"].ravel(), zf, atol=1e-9)
    Ef = npref.objective(pb.D, pb.X, zf.reshape(pb.K, pb.Tz), lam)
    assert oracle.objective(pb.D, pb.X, r["Z"], lam) == pytest.approx(Ef, rel=1e-12)


def test_matches_exhaustive_lasso():
    pb = tiny(K=2, P=2, L=3, T=6, rho=0.4, sigma=0.3, seed=11)
    A = npref.operator(pb.D, pb.T)
    x = pb.X.astype(np.float64).ravel()
    lam = 0.15 * oracle.lambda_max(pb.D, pb.X)
    zb, Eb = npref.brute_force_lasso(A, x, lam)
    assert np.count_nonzero(zb) >= 2
    for r in (oracle.greedy_cd(pb.D, pb.X, lam, 1e-14, max_updates=CAP),
              oracle.locally_greedy_cd(pb.D, pb.X, lam, 1e-14, M=2, mode="phase", max_updates=CAP),
              oracle.locally_greedy_cd(pb.D, pb.X, lam, 1e-14, M=4, mode="random", seed=3, max_updates=CAP)):
        assert r["converged"]
        np.testing.assert_allclose(r["Z"].ravel(), zb, atol=1e-10)
        assert oracle.objective(pb.D, pb.X, r["Z"], lam) == pytest.approx(Eb, rel=1e-12)


def test_kkt_at_solution():
    # coordinate-wise optimality (Theorem A.1): |beta| <= lam where Z == 0,
    # Z == Sh(beta, lam)/n elsewhere
    pb = tiny(K=3, P=2, L=8, T=120, seed=13)
    lam = 0.1 * oracle.lambda_max(pb.D, pb.X)
    r = oracle.greedy_cd(pb.D, pb.X, lam, 1e-12, max_updates=CAP)
    assert r["converged"]
    B = npref.beta_fresh(pb.D, pb.X, r["Z"])
    n = npref.norms(pb.D)
    z = r["Z"]
    assert np.all(np.abs(B[z == 0]) <= lam * (1 + 1e-9))
    gap = np.abs(z - npref.soft(B, lam) / n[:, None])
    assert gap.max() <= 1e-11
    rep = oracle.kkt(B, z, n, lam)
    assert rep["zero_excess"] <= 1e-9 and rep["nonzero_gap"] <= 1e-11


# ---------------------------------------------- Alg. 3 / phase schedule

def test_kkt_report_at_zero_and_after_one_coordinate():
    # Theorem A.1 at Z = 0: beta = D~*X, so the excess over the zero coordinates
    # is lambda_max - lambda, there is no nonzero gap, and the largest |Delta Z|
    # is the step Alg. 1 takes first; flipping X flips beta, not the report.
    pb = tiny()
    n = npref.norms(pb.D)
    lmax = float(np.abs(npref.dtx_fft(pb.D, pb.X)).max())
    lam = 0.5 * lmax
    Z0 = np.zeros((pb.K, pb.Tz))
    first = oracle.greedy_cd(pb.D, pb.X, lam, 1e-12, max_updates=1, trace=1)
    z1 = float(first["trace"]["z_new"][0])
    assert z1 != 0.0
    for X in (pb.X, -pb.X):
        rep = oracle.kkt(oracle.beta_fresh(pb.D, X, Z0), Z0, n, lam)
        assert rep["zero_excess"] == pytest.approx(lmax - lam, rel=1e-12)
        assert rep["nonzero_gap"] == 0.0
        assert rep["max_delta_z"] == pytest.approx(abs(z1), rel=1e-12)
    # that coordinate alone set to 3x its optimum: beta there excludes its own
    # contribution, so its gap is |3 z1 - z1| and it is the only nonzero
    k, t = int(first["trace"]["k"][0]), int(first["trace"]["t"][0])
    Z1 = Z0.copy()
    Z1[k, t] = 3.0 * z1
    rep = oracle.kkt(oracle.beta_fresh(pb.D, pb.X, Z1), Z1, n, lam)
    assert rep["nonzero_gap"] == pytest.approx(2.0 * abs(z1), rel=1e-10)
    assert rep["max_delta_z"] >= rep["nonzero_gap"]


def test_single_segment_equals_greedy_trajectory():
    # M = 1: the locally greedy argmax is the global one (Alg. 3 -> Alg. 1)
    pb = tiny(K=3, P=2, L=6, T=90, seed=17)
    lam = 0.1 * oracle.lambda_max(pb.D, pb.X)
    g = oracle.greedy_cd(pb.D, pb.X, lam, 1e-9, trace=10_000, max_updates=CAP)
    p = oracle.locally_greedy_cd(pb.D, pb.X, lam, 1e-9, M=1, mode="phase", trace=10_000, max_updates=CAP)
    # Alg. 1 applies its final sub-eps update before testing; the schedule tests first
    assert g["n_updates"] == p["n_updates"] + 1
    for key in ("k", "t", "z_old", "z_new"):
        np.testing.assert_array_equal(g["trace"][key][:-1], p["trace"][key])
    assert abs(g["trace"]["z_new"][-1] - g["trace"]["z_old"][-1]) < 1e-9


@pytest.mark.parametrize("M,u", [(3, 0), (5, 1), (8, 3)])
def test_locally_greedy_reaches_greedy_optimum(M, u):
    # Theorem conv_dcp: the locally greedy schedules converge to Z*
    pb = tiny(K=3, P=2, L=6, T=150, seed=19)
    lam = 0.1 * oracle.lambda_max(pb.D, pb.X)
    g = oracle.greedy_cd(pb.D, pb.X, lam, 1e-13, max_updates=CAP)
    Eg = oracle.objective(pb.D, pb.X, g["Z"], lam)
    for mode in ("phase", "random"):
        r = oracle.locally_greedy_cd(pb.D, pb.X, lam, 1e-13, M=M, mode=mode, seed=M,
                                     updates_per_visit=u, max_updates=CAP)
        assert r["converged"]
        np.testing.assert_allclose(r["Z"], g["Z"], atol=1e-10)
        assert oracle.objective(pb.D, pb.X, r["Z"], lam) == pytest.approx(Eg, rel=1e-13)


def test_one_update_per_sweep_reaches_greedy_optimum():
    # Theorem conv_dcp with the slowest schedule: one segment, one update per
    # visit, so every sweep applies a single update until none is left
    pb = tiny(K=3, P=2, L=6, T=60, seed=29)
    lam = 0.1 * oracle.lambda_max(pb.D, pb.X)
    g = oracle.greedy_cd(pb.D, pb.X, lam, 1e-13, max_updates=CAP)
    r = oracle.locally_greedy_cd(pb.D, pb.X, lam, 1e-13, M=1, mode="phase",
                                 updates_per_visit=1, max_updates=CAP)
    assert r["converged"] and r["sweeps"] == r["n_updates"] + 1
    np.testing.assert_allclose(r["Z"], g["Z"], atol=1e-10)


def test_segments_partition_and_phases_are_disjoint():
    # Sec. 2.2 segments; co-active segments' update windows [s-L+1, e+L-1) never meet
    rng = np.random.default_rng(0)
    cases = [(199_937, M, 64) for M in (64, 256, 1024, 3072)] + [(1985, 10, 16), (7, 7, 3)]
    cases += [(int(rng.integers(1, 3000)), 0, int(rng.integers(1, 70))) for _ in range(40)]
    for Tz, M, L in cases:
        if M == 0:
            M = int(rng.integers(1, Tz + 1))
        starts = [oracle.segment_start(Tz, M, m) for m in range(M + 1)]
        assert starts[0] == 0 and starts[-1] == Tz
        assert all(b > a for a, b in zip(starts, starts[1:]))
        c = oracle.phase_count(Tz, M, L)
        assert 1 <= c <= M
        for m in range(M):
            for m2 in range(m + c, min(M, m + 4 * c), c):
                assert starts[m + 1] + L - 1 <= starts[m2] - (L - 1), (Tz, M, L, m, m2)
        if M > 1 and L > 1:
            # one phase fewer would let two co-active windows overlap somewhere
            widths = np.diff(starts)
            assert (c - 2) * widths.min() < 2 * L - 2 or c == M


# ------------------------------------------------------- Eq. interf (algebra)

def test_interference_cost_formula():
    # Prop. A.2: two simultaneous optimal updates change E by
    # dE0 + dE1 - S_{k0,k1}[t0-t1] dZ0 dZ1 (with dZ = Z - Z').  Eq. interf in
    # Sec. 2.2 prints the lag as t1-t0; with S_{k,l}[t] = S_{l,k}[-t] that is
    # the same term only with the atom indices swapped, and the appendix
    # derivation fixes it as written here.
    pb = tiny(K=3, P=2, L=6, T=60, seed=23)
    lam = 0.05 * float(np.abs(npref.dtx_fft(pb.D, pb.X)).max())
    S = npref.crosscorr(pb.D)
    n = npref.norms(pb.D)
    rng = np.random.default_rng(4)
    Z = rng.standard_normal((pb.K, pb.Tz)) * (rng.random((pb.K, pb.Tz)) < 0.2)
    L = pb.L
    for _ in range(20):
        k0, k1 = rng.integers(0, pb.K, 2)
        t0 = int(rng.integers(0, pb.Tz))
        t1 = int(np.clip(t0 + rng.integers(-(L - 1), L), 0, pb.Tz - 1))
        if (k0, t0) == (k1, t1):
            continue
        B = npref.beta_fresh(pb.D, pb.X, Z)
        u0 = npref.soft(B[k0, t0], lam) / n[k0]
        u1 = npref.soft(B[k1, t1], lam) / n[k1]
        E = npref.objective(pb.D, pb.X, Z, lam)

        def with_(pairs):
            Y = Z.copy()
            for (k, t, v) in pairs:
                Y[k, t] = v
            return npref.objective(pb.D, pb.X, Y, lam)

        dE0 = E - with_([(k0, t0, u0)])
        dE1 = E - with_([(k1, t1, u1)])
        dE01 = E - with_([(k0, t0, u0), (k1, t1, u1)])
        dz0, dz1 = Z[k0, t0] - u0, Z[k1, t1] - u1
        inter = S[k0, k1, (t0 - t1) + L - 1] * dz0 * dz1
        assert dE01 == pytest.approx(dE0 + dE1 - inter, abs=1e-10 * max(1, E))
