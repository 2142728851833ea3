"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Bars (the solver's stated tolerances):
  * relative objective gap (E_gpu - E_ref) / E_ref <= 1e-5,
  * ||Z_gpu - Z_ref||_inf <= 1e-4 ||Z_ref||_inf,
  * identical support outside |z| < 1e-6: every coordinate that is at least
    1e-6 in magnitude in one solution is nonzero with the same sign in the
    other.
The reference Z_ref is the oracle's solution at eps = 1e-10 (the unique
minimiser up to FP64 rounding); both sides get the same seeded inputs and the
same lambda (computed by the oracle).  Element-wise checks of the setup
kernels use error bounds derived from FP32 compensated summation.
"""
import numpy as np
import pytest

import oracle
from paper_1705_10087_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

U = 2.0 ** -24  # unit roundoff of float32


@pytest.fixture(scope="module")
def capi():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1705_10087_gb300 import build, capi as c
    build.build()
    c.load()
    return c


def cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a, np.float32)).cuda()


def gpu_solve(capi, pb, lam, tol, M=0, u=0, max_updates=1 << 40, Z0=None, host=False,
              max_resyncs=-1):
    opts = capi.make_opts(segments=M, updates_per_visit=u, max_resyncs=max_resyncs)
    D = pb.D if host else cuda(pb.D)
    X = pb.X if host else cuda(pb.X)
    h = capi.csc_setup(D, opts)
    try:
        capi.csc_init(h, X, lam, None if Z0 is None else (Z0 if host else cuda(Z0)))
        beta0 = None
        if Z0 is None:  # cold start: beta = r = D~*X as the library computed it
            b = torch.zeros((pb.K, pb.Tz), dtype=torch.float32, device="cuda")
            capi.csc_get_beta(h, b)
            beta0 = b.cpu().numpy()
        Zo = np.zeros((pb.K, pb.Tz), np.float32) if host else torch.zeros(
            (pb.K, pb.Tz), dtype=torch.float32, device="cuda")
        status, E, st = capi.csc_solve(h, tol, max_updates, Zo)
        beta = torch.zeros((pb.K, pb.Tz), dtype=torch.float32, device="cuda")
        capi.csc_get_beta(h, beta)
        trace = capi.csc_get_trace(h)
        lmax = capi.csc_lambda_max(h)
    finally:
        capi.csc_destroy(h)
    Z = Zo if host else Zo.cpu().numpy()
    return dict(Z=Z, E=E, stats=st, status=status, beta=beta.cpu().numpy(), trace=trace,
                lambda_max=lmax, beta0=beta0)


def assert_parity(Z, E, Zr, Er, tau=1e-6):
    gap = (E - Er) / Er
    assert gap <= 1e-5, gap
    assert gap >= -1e-9, gap
    zinf = np.abs(Zr).max()
    assert np.abs(Z - Zr).max() <= 1e-4 * zinf, np.abs(Z - Zr).max()
    big = (np.abs(Z) >= tau) | (np.abs(Zr) >= tau)
    assert np.all(np.sign(Z[big]) == np.sign(Zr[big])), int(
        (np.sign(Z[big]) != np.sign(Zr[big])).sum())


# ------------------------------------------------------------- problems

SHORT = synth.WORKLOADS["short_P1_K5_L16_T2000"]
LONG = synth.WORKLOADS["long_P7_K25_L64_T200000"]


@pytest.fixture(scope="module")
def short():
    pb = synth.make_workload("short_P1_K5_L16_T2000", seed=0)
    lam = 0.1 * oracle.lambda_max(pb.D, pb.X)
    ref = oracle.greedy_cd(pb.D, pb.X, lam, 1e-10)
    assert ref["converged"]
    return pb, lam, ref, oracle.objective(pb.D, pb.X, ref["Z"], lam)


@pytest.fixture(scope="module")
def long_small():
    # the long-signal recipe at T = 20,000: many tiles and a ragged tail
    pb = synth.make_workload("long_P7_K25_L64_T200000", seed=1, T=20_000)
    lam = 0.1 * oracle.lambda_max(pb.D, pb.X)
    ref = oracle.locally_greedy_cd(pb.D, pb.X, lam, 1e-10, M=64, mode="phase")
    assert ref["converged"]
    return pb, lam, ref, oracle.objective(pb.D, pb.X, ref["Z"], lam)


@pytest.fixture(scope="module")
def long_full():
    pb = synth.make_workload("long_P7_K25_L64_T200000", seed=0)
    lam = 0.1 * oracle.lambda_max(pb.D, pb.X)
    ref = oracle.locally_greedy_cd(pb.D, pb.X, lam, 1e-10, M=1024, mode="phase")
    assert ref["converged"]
    return pb, lam, ref, oracle.objective(pb.D, pb.X, ref["Z"], lam)


# ------------------------------------------------------- setup kernels

def test_dtd_and_norms_elementwise(capi):
    for (K, P, L) in [(5, 1, 16), (25, 7, 64), (3, 2, 1), (25, 1, 200)]:
        D = synth.make_dictionary(K, P, L, seed=K + L)
        h = capi.csc_setup(cuda(D))
        C = torch.zeros((K, K, 2 * L - 1), dtype=torch.float32, device="cuda")
        n = torch.zeros(K, dtype=torch.float32, device="cuda")
        capi.csc_get_dtd(h, C, n)
        capi.csc_destroy(h)
        S = oracle.crosscorr(D)          # S[k,l,s] ; the library stores C[k0][k][s] = S[k][k0][s]
        want = np.transpose(S, (1, 0, 2))
        bound = oracle.crosscorr(np.abs(D))  # sum of |terms|
        err = np.abs(C.cpu().numpy() - want)
        assert np.all(err <= 10 * U * np.transpose(bound, (1, 0, 2)) + 2 * U * np.abs(want)), err.max()
        np.testing.assert_allclose(n.cpu().numpy(), oracle.norms(D), rtol=4 * U * L * P)


@pytest.mark.parametrize("K,P,L,T", [(5, 1, 16, 2000), (25, 7, 64, 20_000), (3, 2, 5, 5),
                                     (25, 1, 200, 3001), (1, 1, 1, 700)])
def test_dtx_elementwise(capi, K, P, L, T):
    # the FP32 CUDA-core kernel (init_mode 3); the tensor-core kernel has its own
    # bound in tests/test_gpu_dtx_tc.py
    pb = synth.make_problem(K=K, P=P, L=L, T=T, rho=0.01, sigma=0.1, seed=2)
    h = capi.csc_setup(cuda(pb.D), capi.make_opts(init_mode=3))
    capi.csc_init(h, cuda(pb.X), 1.0)
    beta = torch.zeros((K, pb.Tz), dtype=torch.float32, device="cuda")
    capi.csc_get_beta(h, beta)
    lmax = capi.csc_lambda_max(h)
    capi.csc_destroy(h)
    want = oracle.dtx(pb.D, pb.X)
    bound = oracle.dtx(np.abs(pb.D), np.abs(pb.X))
    err = np.abs(beta.cpu().numpy() - want)
    assert np.all(err <= 10 * U * bound + 2 * U * np.abs(want)), err.max()
    assert lmax == pytest.approx(np.abs(want).max(), rel=4 * U)


# ------------------------------------------------------------ solves

@pytest.mark.parametrize("M", [1, 10])
@pytest.mark.parametrize("tol", [1e-6, 1e-7])
def test_short_signal_parity(capi, short, M, tol):
    # 1e-6 is the workload's stopping rule; 1e-7 is below the FP32 resolution of
    # the largest beta and must still end at the optimum, not drift
    pb, lam, ref, Er = short
    r = gpu_solve(capi, pb, lam, tol, M=M)
    assert r["status"] == 0 and r["stats"]["converged"] == 1
    assert_parity(r["Z"], r["E"], ref["Z"], Er)
    # the GPU's FP64 objective is E(Z_gpu) by the definition
    assert r["E"] == pytest.approx(oracle.objective(pb.D, pb.X, r["Z"], lam), rel=1e-12)


def test_short_signal_at_config_tolerance(capi, short):
    # the workload's own stopping rule, max |Delta Z| < 1e-6 (Alg. 1)
    pb, lam, ref, Er = short
    r = gpu_solve(capi, pb, lam, SHORT["tol"], M=10)
    assert r["status"] == 0
    o = oracle.locally_greedy_cd(pb.D, pb.X, lam, SHORT["tol"], M=10, mode="phase")
    Eo = oracle.objective(pb.D, pb.X, o["Z"], lam)
    assert (r["E"] - Er) / Er <= 1e-5 and (Eo - Er) / Er <= 1e-5
    assert np.abs(r["Z"] - ref["Z"]).max() <= 1e-4 * np.abs(ref["Z"]).max()
    # optimality at the configured tolerance, against a fresh FP64 beta
    B = oracle.beta_fresh(pb.D, pb.X, r["Z"])
    assert oracle.kkt(B, r["Z"], oracle.norms(pb.D), lam)["max_delta_z"] < 2 * SHORT["tol"]


@pytest.mark.parametrize("M,u", [(64, 0), (16, 0), (64, 1), (313, 0), (1000, 0)])
def test_long_signal_reduced_parity(capi, long_small, M, u):
    pb, lam, ref, Er = long_small
    r = gpu_solve(capi, pb, lam, LONG["tol"], M=M, u=u)
    assert r["status"] == 0, r["stats"]
    assert_parity(r["Z"], r["E"], ref["Z"], Er)
    # beta kept by the kernels equals the definition at the returned Z
    B = oracle.beta_fresh(pb.D, pb.X, r["Z"])
    assert np.abs(r["beta"] - B).max() <= 1e-5


_BETA0 = {}


def _exact_beta0(pb):
    """D~*X from the FP64 oracle (computed once per problem)."""
    key = (pb.seed, pb.X.shape)
    if key not in _BETA0:
        _BETA0[key] = oracle.dtx(pb.D, pb.X)
    return _BETA0[key]


@pytest.mark.slow
@pytest.mark.parametrize("M,u", [(M, 0) for M in LONG["segments"]] + [(1024, 24)])
def test_long_signal_full_size_parity(capi, long_full, M, u):
    # the full long-signal workload over the segment sweep, and in the launch
    # configuration the benchmark times (M = 1024, 24 updates per visit)
    pb, lam, ref, Er = long_full
    r = gpu_solve(capi, pb, lam, LONG["tol"], M=M, u=u)
    assert r["status"] == 0, r["stats"]
    assert_parity(r["Z"], r["E"], ref["Z"], Er)
    st = r["stats"]
    assert st["kkt_zero_excess"] <= 1e-5 and st["kkt_nonzero_gap"] <= 1e-5
    # objective trace (Prop. A.1 per update, from E(0) = |X|^2 / 2) agrees with the
    # final FP64 objective.  The decreases are those of the problem whose beta0
    # is the one the library computed (the state r is exact for it after each
    # resync), whose objective at Z is E(Z) - <Z, beta0_computed - D~*X>.
    tr = r["trace"]
    offset = float(np.sum(r["Z"].astype(np.float64) *
                          (r["beta0"].astype(np.float64) - _exact_beta0(pb))))
    assert tr["E_start"] - tr["decrease"].sum() == pytest.approx(r["E"] - offset, rel=1e-6)
    assert tr["updates"].sum() == st["updates"]


# ------------------------------------------------------------ edge cases

def test_lambda_above_lambda_max(capi, short):
    pb = short[0]
    lmax = oracle.lambda_max(pb.D, pb.X)
    r = gpu_solve(capi, pb, lmax * 1.001, 1e-7, M=10)
    assert r["status"] == 0 and r["stats"]["updates"] == 0
    assert not r["Z"].any()
    assert r["lambda_max"] == pytest.approx(lmax, rel=1e-6)


def test_single_time_position_closed_form(capi):
    # T = L: Tz = 1; disjoint channels make the Gram diagonal (Eq. pb_coord closed form)
    K, L = 4, 9
    rng = np.random.default_rng(5)
    D = np.zeros((K, K, L), np.float32)
    for k in range(K):
        D[k, k] = rng.standard_normal(L) * (0.5 + k)
    X = (rng.standard_normal((K, L)) * 3).astype(np.float32)
    pb = synth.Problem(D=D, Z_true=np.zeros((K, 1), np.float32), X=X, seed=0, rho=0, sigma=0)
    lam = 0.7
    r = gpu_solve(capi, pb, lam, 1e-7, M=1)
    want = np.array([np.sign(D[k, k] @ X[k]) * max(abs(float(D[k, k].astype(np.float64) @ X[k])) - lam, 0)
                     / float((D[k, k].astype(np.float64) ** 2).sum()) for k in range(K)])
    np.testing.assert_allclose(r["Z"][:, 0], want, rtol=1e-5, atol=1e-6)


def test_one_sample_segments(capi):
    # M = Tz: segments of width 1, many phases
    pb = synth.make_problem(K=2, P=1, L=4, T=40, rho=0.1, sigma=0.05, seed=8)
    lam = 0.1 * oracle.lambda_max(pb.D, pb.X)
    ref = oracle.greedy_cd(pb.D, pb.X, lam, 1e-10)
    r = gpu_solve(capi, pb, lam, 1e-7, M=pb.Tz)
    assert r["stats"]["phases"] == oracle.phase_count(pb.Tz, pb.Tz, pb.L)
    assert_parity(r["Z"], r["E"], ref["Z"], oracle.objective(pb.D, pb.X, ref["Z"], lam))


def test_single_atom_single_channel(capi):
    pb = synth.make_problem(K=1, P=1, L=8, T=3000, rho=0.02, sigma=0.05, seed=9)
    lam = 0.1 * oracle.lambda_max(pb.D, pb.X)
    ref = oracle.greedy_cd(pb.D, pb.X, lam, 1e-10)
    r = gpu_solve(capi, pb, lam, 1e-7, M=37)
    assert_parity(r["Z"], r["E"], ref["Z"], oracle.objective(pb.D, pb.X, ref["Z"], lam))


def test_max_updates_reports_not_converged(capi, short):
    pb, lam, ref, Er = short
    r = gpu_solve(capi, pb, lam, 1e-7, M=10, max_updates=20)
    assert r["status"] == 1 and r["stats"]["converged"] == 0
    assert 20 <= r["stats"]["updates"] < 20 + 10 * (1 << 20)
    assert r["E"] == pytest.approx(oracle.objective(pb.D, pb.X, r["Z"], lam), rel=1e-12)
    assert r["E"] < r["trace"]["E_start"]


def test_host_pointers_match_device_pointers(capi, short):
    pb, lam, ref, Er = short
    a = gpu_solve(capi, pb, lam, 1e-7, M=10)
    b = gpu_solve(capi, pb, lam, 1e-7, M=10, host=True)
    np.testing.assert_array_equal(a["Z"], b["Z"])
    assert a["E"] == b["E"]


def test_deterministic(capi, long_small):
    pb, lam, ref, Er = long_small
    a = gpu_solve(capi, pb, lam, 1e-7, M=64)
    b = gpu_solve(capi, pb, lam, 1e-7, M=64)
    np.testing.assert_array_equal(a["Z"], b["Z"])


@pytest.mark.parametrize("T,M", [(20_000, 64), (5_131, 10)])
def test_solve_objective_equals_a_fresh_one_bitwise(capi, T, M):
    # the objective a solve returns is computed from the nonzero lists of its
    # last resync; csc_objective on the same Z lists Z itself: the same sums in
    # the same order, so the same double; both match the oracle's E of that Z
    pb = synth.make_workload("long_P7_K25_L64_T200000", seed=2, T=T)
    lam = 0.1 * oracle.lambda_max(pb.D, pb.X)
    h = capi.csc_setup(cuda(pb.D), capi.make_opts(segments=M))
    try:
        capi.csc_init(h, cuda(pb.X), lam)
        Z = torch.zeros((pb.K, pb.Tz), dtype=torch.float32, device="cuda")
        status, E, st = capi.csc_solve(h, 1e-6, 1 << 40, Z)
        assert status == capi.CSC_OK
        assert capi.csc_objective(h, Z) == E
    finally:
        capi.csc_destroy(h)
    Er = oracle.objective(pb.D, pb.X, Z.cpu().numpy().astype(np.float64), lam)
    assert abs(E - Er) <= 1e-12 * abs(Er)


def test_warm_start_from_optimum(capi, short):
    # csc_init with Z0: beta = D~*X - DtD Z0 + n Z0 in FP64 (the beta definition)
    pb, lam, ref, Er = short
    Z0 = ref["Z"].astype(np.float32)
    r = gpu_solve(capi, pb, lam, 1e-6, M=10, Z0=Z0)
    assert r["stats"]["updates"] <= 5
    B = oracle.beta_fresh(pb.D, pb.X, Z0)
    assert np.abs(r["beta"] - B).max() <= 1e-5
    assert_parity(r["Z"], r["E"], ref["Z"], Er)


def test_kkt_report_of_any_Z(capi, long_small):
    """csc_kkt: the optimality report (Theorem A.1) of a caller's Z against the
    oracle's FP64 report of the same Z, on host and device pointers; of the
    solve's own Z it is the report the solve returned, and it leaves the
    handle's state alone."""
    pb, lam, ref, Er = long_small
    h = capi.csc_setup(cuda(pb.D), capi.make_opts(segments=64))
    try:
        capi.csc_init(h, cuda(pb.X), lam)
        Zd = torch.zeros((pb.K, pb.Tz), dtype=torch.float32, device="cuda")
        status, E, st = capi.csc_solve(h, 1e-7, 1 << 40, Zd)
        b_before = torch.zeros_like(Zd)
        capi.csc_get_beta(h, b_before)
        own = capi.csc_kkt(h, Zd)
        Z = Zd.cpu().numpy()
        rng = np.random.default_rng(3)
        Zp = Z.copy()
        mask = rng.random(Z.shape) < 0.01
        Zp[mask] += rng.standard_normal(int(mask.sum())).astype(np.float32)
        pert = capi.csc_kkt(h, Zp)
        again = capi.csc_kkt(h, Zd)
        b_after = torch.zeros_like(Zd)
        capi.csc_get_beta(h, b_after)
    finally:
        capi.csc_destroy(h)
    assert status == 0
    assert torch.equal(b_before, b_after)
    assert again == own
    for key, sk in (("zero_excess", "kkt_zero_excess"), ("nonzero_gap", "kkt_nonzero_gap"),
                    ("max_delta_z", "max_delta_z")):
        assert own[key] == pytest.approx(st[sk], rel=1e-6, abs=1e-12)
    n = oracle.norms(pb.D)
    for Zc, got in ((Z, own), (Zp, pert)):
        B = oracle.beta_fresh(pb.D, pb.X, Zc)
        want = oracle.kkt(B, Zc, n, lam)
        # beta in float32 from an FP64-accurate residual and the FP32 D~*X
        tol = 1e-5 * float(np.abs(B).max())
        for key in want:
            assert abs(got[key] - want[key]) <= tol, (key, got[key], want[key])
    assert pert["max_delta_z"] > 1e3 * max(own["max_delta_z"], 1e-9)


def test_invalid_arguments_raise(capi):
    D = cuda(synth.make_dictionary(3, 1, 8, seed=0))
    h = capi.csc_setup(D)
    try:
        with pytest.raises(capi.CscError):
            capi.csc_solve(h, 1e-6)          # before csc_init
        with pytest.raises(capi.CscError):
            capi.csc_init(h, cuda(np.zeros((1, 5), np.float32)), 1.0)   # T < L
        with pytest.raises(capi.CscError):
            capi.csc_init(h, cuda(np.zeros((1, 50), np.float32)), -1.0)  # lambda <= 0
        capi.csc_init(h, cuda(np.ones((1, 50), np.float32)), 0.5)
        with pytest.raises(capi.CscError):
            capi.csc_solve(h, 0.0)
    finally:
        capi.csc_destroy(h)


def test_status_after_the_last_resync_is_the_exact_check(capi):
    """After the last resync allowed, csc_solve's status is the exact check's:
    with one resync allowed this problem's float32 loop settles twice while
    the refreshed state still has a coordinate above tol, so the solve must
    say CSC_NOT_CONVERGED (not a limit: few sweeps, few updates); with two
    resyncs allowed the third refresh passes and the solve converges.  tol is
    below the float32 floor, where only the refresh can tell."""
    pb = synth.make_problem(K=25, P=7, L=64, T=20_000, rho=0.005, sigma=0.1, seed=1)
    D, X = cuda(pb.D), cuda(pb.X)
    tol, max_sweeps = 1e-9, 2000
    out = {}
    for mr in (1, 2):
        h = capi.csc_setup(D, capi.make_opts(max_resyncs=mr, updates_per_visit=24,
                                             max_sweeps=max_sweeps))
        try:
            capi.csc_init(h, X, 1.0)
            lam = 0.1 * capi.csc_lambda_max(h)
            capi.csc_init(h, X, lam)
            out[mr] = capi.csc_solve(h, tol, 1 << 40)
        finally:
            capi.csc_destroy(h)
    status, E, st = out[1]
    assert status == capi.CSC_NOT_CONVERGED and st["converged"] == 0, st
    assert st["resyncs"] == 2 and st["sweeps"] < max_sweeps, st  # the check, not a limit
    assert st["max_delta_z"] >= tol
    status2, E2, st2 = out[2]
    assert status2 == capi.CSC_OK and st2["converged"] == 1, st2
    assert E2 <= E * (1 + 1e-12)


@pytest.mark.parametrize("tps", [32, 128])
@pytest.mark.parametrize("M,u", [(64, 0), (313, 24), (1000, 1)])
def test_both_phase_kernel_forms_match_the_oracle(capi, long_small, M, u, tps):
    """One warp per segment and a block per segment (csc_opts.threads_per_segment)
    run the same coordinate steps: both meet the parity bars."""
    pb, lam, ref, Er = long_small
    opts = capi.make_opts(segments=M, updates_per_visit=u, threads_per_segment=tps)
    h = capi.csc_setup(cuda(pb.D), opts)
    try:
        capi.csc_init(h, cuda(pb.X), lam)
        Z = torch.zeros((pb.K, pb.Tz), dtype=torch.float32, device="cuda")
        status, E, st = capi.csc_solve(h, LONG["tol"], 1 << 40, Z)
    finally:
        capi.csc_destroy(h)
    assert status == 0, st
    assert_parity(Z.cpu().numpy(), E, ref["Z"], Er)


@pytest.mark.slow
def test_warp_form_full_size_parity(capi, long_full):
    pb, lam, ref, Er = long_full
    r = gpu_solve(capi, pb, lam, LONG["tol"], M=1024, u=24)  # automatic form
    assert r["status"] == 0
    assert_parity(r["Z"], r["E"], ref["Z"], Er)
    opts = capi.make_opts(segments=1024, updates_per_visit=24, threads_per_segment=128)
    h = capi.csc_setup(cuda(pb.D), opts)
    try:
        capi.csc_init(h, cuda(pb.X), lam)
        Z = torch.zeros((pb.K, pb.Tz), dtype=torch.float32, device="cuda")
        status, E, st = capi.csc_solve(h, LONG["tol"], 1 << 40, Z)
    finally:
        capi.csc_destroy(h)
    assert status == 0
    assert_parity(Z.cpu().numpy(), E, ref["Z"], Er)
