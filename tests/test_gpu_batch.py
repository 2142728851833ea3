"""Batches of signals (csc_init_batch): every signal's result must be that of
solving it alone, checked against the FP64 oracle run on each signal by itself.

Same bars as tests/test_gpu_parity.py, per signal: relative objective gap
<= 1e-5, ||Z - Z_ref||_inf <= 1e-4 ||Z_ref||_inf, identical support outside
|z| < 1e-6.  The columns that straddle two signals must stay exactly 0.
"""
import numpy as np
import pytest

import oracle
from paper_1705_10087_gb300 import batch, synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


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


def assert_parity(Z, E, Zr, Er, tau=1e-6):
    gap = (E - Er) / Er
    assert gap <= 1e-5, gap
    assert gap >= -1e-9, gap
    zinf = np.abs(Zr).max()
    assert np.abs(Z - Zr).max() <= 1e-4 * zinf, (np.abs(Z - Zr).max(), zinf)
    big = (np.abs(Z) >= tau) | (np.abs(Zr) >= tau)
    assert np.all(np.sign(Z[big]) == np.sign(Zr[big]))


def oracle_solution(D, X, lam):
    """Z* of one signal: locally greedy CD to eps = 1e-10 (any exact method agrees)."""
    Tz = X.shape[1] - D.shape[2] + 1
    M = max(1, Tz // (2 * D.shape[2] - 2)) if D.shape[2] > 1 else 1
    ref = oracle.locally_greedy_cd(D, X, lam, 1e-10, M=min(M, 64), mode="phase")
    assert ref["converged"]
    return ref["Z"], oracle.objective(D, X, ref["Z"], lam)


def solve_batch(capi, D, Xs, lams, tol=1e-6, width=0, u=0, Z0=None, host=False,
                launch_mode=0):
    X, T = batch.pack(Xs)
    K, L = D.shape[0], D.shape[2]
    h = capi.csc_setup(D if host else cuda(D),
                       capi.make_opts(segment_width=width, updates_per_visit=u,
                                      launch_mode=launch_mode))
    try:
        capi.csc_init_batch(h, X if host else cuda(X), T, lams,
                            None if Z0 is None else (Z0 if host else cuda(Z0)))
        lmax = capi.csc_lambda_max_batch(h, len(Xs))
        Tz = int(T.sum()) - L + 1
        Zo = np.zeros((K, Tz), np.float32)
        status, E, st = capi.csc_solve(h, tol, 1 << 40, Zo)
        Es = capi.csc_get_objectives(h, len(Xs))
    finally:
        capi.csc_destroy(h)
    return dict(Z=Zo, T=T, E=E, Es=Es, stats=st, status=status, lmax=lmax)


def check_batch(res, D, Xs, lams, refs):
    L = D.shape[2]
    T = res["T"]
    assert res["status"] == 0 and res["stats"]["converged"] == 1
    # the columns between signals belong to no problem and stay exactly 0
    assert not np.any(res["Z"][:, batch.straddle_mask(T, L)])
    Zs = batch.unpack_Z(res["Z"], T, L)
    for i, (X, lam, (Zr, Er)) in enumerate(zip(Xs, lams, refs)):
        Ei = oracle.objective(D, X, Zs[i], lam)
        # the library's per-signal FP64 objective of its own Z
        assert abs(res["Es"][i] - Ei) <= 1e-9 * Ei, (i, res["Es"][i], Ei)
        if not np.any(Zr):
            assert not np.any(Zs[i]), i          # lambda >= lambda_max: Z* = 0 exactly
            continue
        assert_parity(Zs[i], Ei, Zr, Er)
    assert abs(res["E"] - res["Es"].sum()) <= 1e-12 * res["E"]


def short_batch():
    """Short single-channel signals of uneven length (Tz from 1 to 1985) sharing
    one dictionary; one signal has lambda above its lambda_max."""
    w = synth.WORKLOADS["short_P1_K5_L16_T2000"]
    D = synth.make_dictionary(w["K"], w["P"], w["L"], seed=0)
    Ts = [2000, 16, 17, 31, 777, 2000, 45]
    pbs = [synth.make_problem(K=w["K"], P=w["P"], L=w["L"], T=T, rho=w["rho"],
                              sigma=w["sigma"], seed=100 + i, D=D) for i, T in enumerate(Ts)]
    Xs = [pb.X for pb in pbs]
    lmax = [oracle.lambda_max(D, X) for X in Xs]
    lams = [0.1 * m for m in lmax]
    lams[3] = 2.0 * lmax[3]
    return D, Xs, lams, lmax


@pytest.fixture(scope="module")
def short_refs():
    D, Xs, lams, lmax = short_batch()
    return D, Xs, lams, lmax, [oracle_solution(D, X, lam) for X, lam in zip(Xs, lams)]


def test_batch_short_signals_match_oracle(capi, short_refs):
    D, Xs, lams, lmax, refs = short_refs
    res = solve_batch(capi, D, Xs, lams)
    check_batch(res, D, Xs, lams, refs)
    # lambda_max of each signal: max |D~ * X_i| in FP32 with compensated sums
    np.testing.assert_allclose(res["lmax"], lmax, rtol=1e-5)


def test_kkt_report_of_a_batch(capi, short_refs):
    """csc_kkt over a batch: each signal against its own lambda and its own
    columns of the packed Z; the maxima over the signals of the oracle's FP64
    report per signal."""
    D, Xs, lams, lmax, refs = short_refs
    X, T = batch.pack(Xs)
    L = D.shape[2]
    Zp = batch.pack_Z([Zr.astype(np.float32) for Zr, _ in refs], L)
    rng = np.random.default_rng(5)
    mask = rng.random(Zp.shape) < 0.02
    mask[:, batch.straddle_mask(T, L)] = False
    Zp[mask] += rng.standard_normal(int(mask.sum())).astype(np.float32)
    h = capi.csc_setup(cuda(D))
    try:
        capi.csc_init_batch(h, cuda(X), T, lams)
        got = capi.csc_kkt(h, cuda(Zp))
    finally:
        capi.csc_destroy(h)
    n = oracle.norms(D)
    want = {"zero_excess": 0.0, "nonzero_gap": 0.0, "max_delta_z": 0.0}
    scale = 0.0
    for Xi, lam, Zi in zip(Xs, lams, batch.unpack_Z(Zp, T, L)):
        B = oracle.beta_fresh(D, Xi, Zi)
        r = oracle.kkt(B, Zi, n, lam)
        for key in want:
            want[key] = max(want[key], r[key])
        scale = max(scale, float(np.abs(B).max()))
    for key in want:
        assert abs(got[key] - want[key]) <= 1e-5 * scale, (key, got[key], want[key])


def test_batch_host_pointers(capi, short_refs):
    D, Xs, lams, lmax, refs = short_refs
    res = solve_batch(capi, D, Xs, lams, host=True)
    check_batch(res, D, Xs, lams, refs)


@pytest.mark.parametrize("width,u", [(0, 0), (30, 4), (500, 0), (1, 1)])
def test_batch_segment_widths(capi, short_refs, width, u):
    # width 1: one segment per column (many phases); 500: few segments per signal
    D, Xs, lams, lmax, refs = short_refs
    res = solve_batch(capi, D, Xs, lams, width=width, u=u)
    check_batch(res, D, Xs, lams, refs)


@pytest.fixture(scope="module")
def long_refs():
    # the long multichannel recipe at uneven lengths: Tz = 1 (T = L), Tz = 67
    # (one segment, narrower than 2L - 2), and several tiles with ragged tails
    w = synth.WORKLOADS["long_P7_K25_L64_T200000"]
    D = synth.make_dictionary(w["K"], w["P"], w["L"], seed=7)
    Ts = [5000, 12_345, 64, 130, 20_000, 3001]
    pbs = [synth.make_problem(K=w["K"], P=w["P"], L=w["L"], T=T, rho=w["rho"],
                              sigma=w["sigma"], seed=200 + i, D=D) for i, T in enumerate(Ts)]
    Xs = [pb.X for pb in pbs]
    lams = [0.1 * oracle.lambda_max(D, X) for X in Xs]
    return D, Xs, lams, [oracle_solution(D, X, lam) for X, lam in zip(Xs, lams)]


@pytest.mark.parametrize("u", [0, 24])
def test_batch_long_recipe_matches_oracle(capi, long_refs, u):
    D, Xs, lams, refs = long_refs
    res = solve_batch(capi, D, Xs, lams, u=u)
    check_batch(res, D, Xs, lams, refs)


def test_batch_of_one_is_csc_init(capi, long_refs):
    # a batch of one signal runs exactly the plan and arithmetic of csc_init
    D, Xs, lams, refs = long_refs
    res = solve_batch(capi, D, Xs[4:5], lams[4:5])
    h = capi.csc_setup(cuda(D))
    try:
        capi.csc_init(h, cuda(Xs[4]), lams[4])
        Z = np.zeros_like(res["Z"])
        status, E, st = capi.csc_solve(h, 1e-6, 1 << 40, Z)
    finally:
        capi.csc_destroy(h)
    assert status == 0
    assert np.array_equal(Z, res["Z"])
    assert E == res["E"]


def test_batch_warm_start(capi, long_refs):
    # warm start at the oracle optimum, perturbed: converges back to it
    D, Xs, lams, refs = long_refs
    L = D.shape[2]
    rng = np.random.default_rng(5)
    Zs = [np.where(Zr != 0, Zr * (1 + 0.1 * rng.standard_normal(Zr.shape)), 0.0).astype(np.float32)
          for Zr, _ in refs]
    res = solve_batch(capi, D, Xs, lams, Z0=batch.pack_Z(Zs, L))
    check_batch(res, D, Xs, lams, refs)


def test_set_lambda_continues_from_current_Z(capi, short_refs):
    # regularisation path: solve at 3x lambda, lower it in place, solve again
    D, Xs, lams, lmax, refs = short_refs
    X, T = batch.pack(Xs)
    h = capi.csc_setup(cuda(D))
    try:
        capi.csc_init_batch(h, cuda(X), T, [3.0 * l for l in lams])
        status, _, _ = capi.csc_solve(h, 1e-6)
        assert status == 0
        capi.csc_set_lambda(h, lams)
        Z = np.zeros((D.shape[0], int(T.sum()) - D.shape[2] + 1), np.float32)
        status, E, st = capi.csc_solve(h, 1e-6, 1 << 40, Z)
        Es = capi.csc_get_objectives(h, len(Xs))
    finally:
        capi.csc_destroy(h)
    check_batch(dict(Z=Z, T=T, E=E, Es=Es, stats=st, status=status), D, Xs, lams, refs)


def test_batch_argument_errors(capi):
    D = synth.make_dictionary(3, 1, 8, seed=1)
    h = capi.csc_setup(cuda(D))
    try:
        with pytest.raises(capi.CscError):
            capi.csc_set_lambda(h, [1.0])                     # before csc_init
        X = cuda(np.ones((1, 30), np.float32))
        with pytest.raises(capi.CscError):
            capi.csc_init_batch(h, X, [20, 7, 3], [1.0, 1.0, 1.0])   # T < L
        with pytest.raises(capi.CscError):
            capi.csc_init_batch(h, X, [20, 10], [1.0, 0.0])   # lambda <= 0
        with pytest.raises(capi.CscError):
            capi.csc_init_batch(h, X, [20, 10], [1.0, float("nan")])
        with pytest.raises(ValueError):
            capi.csc_init_batch(h, X, [20, 9], [1.0, 1.0])    # sum T != X columns
        capi.csc_init_batch(h, X, [20, 10], [0.5, 0.5])
        with pytest.raises(capi.CscError):
            capi.csc_set_lambda(h, [0.5, -1.0])
    finally:
        capi.csc_destroy(h)


def test_batch_full_size_sampled(capi):
    """The 512-signal batch (lengths uniform in [1e4, 5e5], P=7, K=25, L=64) at
    full size in one solve, as the benchmark runs it; the two shortest signals
    are checked against the oracle and every signal against the optimality
    report and its own cold-start objective."""
    pbs = synth.make_batch("batch_P7_K25_L64_n512_T10000_500000", seed=0, workers=16)
    D = pbs[0].D
    Xs = [pb.X for pb in pbs]
    X, T = batch.pack(Xs)
    del Xs
    L = D.shape[2]
    Xd = cuda(X)
    h = capi.csc_setup(cuda(D), capi.make_opts(updates_per_visit=24))
    try:
        capi.csc_init_batch(h, Xd, T, np.ones(len(T)))
        lam = 0.1 * capi.csc_lambda_max_batch(h, len(T))
        capi.csc_init_batch(h, Xd, T, lam)
        Zd = torch.zeros((D.shape[0], int(T.sum()) - L + 1), dtype=torch.float32, device="cuda")
        status, E, st = capi.csc_solve(h, 1e-6, 1 << 40, Zd)
        Es = capi.csc_get_objectives(h, len(T))
    finally:
        capi.csc_destroy(h)
    assert status == 0 and st["converged"] == 1
    # below tol, or below the float32 resolution of the state (csc_solve's
    # stopping rule): the representable change fl(z + d) - z is held to
    # 2^-21 |r| / n + 2^-22 |z| (|r| <= lambda at the optimum), and the
    # reported change d itself exceeds it by at most half an ulp of z, 2^-24 |z|
    zmax = float(Zd.abs().max())
    floor_ = 2.0 ** -21 * lam.max() + (2.0 ** -22 + 2.0 ** -24) * zmax
    assert st["max_delta_z"] < max(1e-6, floor_) * 1.01
    assert st["kkt_zero_excess"] <= 1e-6 * lam.max()
    a = batch.offsets(T)
    sample = np.argsort(T)[:2]
    for i in sample:
        Zi = Zd[:, int(a[i]):int(a[i + 1]) - L + 1].cpu().numpy()
        Xi = X[:, a[i]:a[i + 1]]
        # lambda of the library (float32 lambda_max) is passed to the oracle as is
        Zr, Er = oracle_solution(D, Xi, float(lam[i]))
        Ei = oracle.objective(D, Xi, Zi, float(lam[i]))
        assert abs(Es[i] - Ei) <= 1e-9 * Ei
        assert_parity(Zi, Ei, Zr, Er)
    # every objective below E(0) = |X_i|^2 / 2
    E0 = np.array([0.5 * np.square(X[:, a[i]:a[i + 1]].astype(np.float64)).sum()
                   for i in range(len(T))])
    assert np.all(Es < E0)
    assert not torch.any(Zd[:, torch.from_numpy(batch.straddle_mask(T, L)).cuda()])


def test_autotune_restores_state_and_keeps_parity(capi, long_refs):
    D, Xs, lams, refs = long_refs
    X, T = batch.pack(Xs)
    K, L = D.shape[0], D.shape[2]
    Tz = int(T.sum()) - L + 1
    h = capi.csc_setup(cuda(D))
    try:
        capi.csc_init_batch(h, cuda(X), T, lams)
        E0 = capi.csc_objective(h, np.zeros((K, Tz), np.float32))
        r = capi.csc_autotune(h, 1e-6)
        assert r["candidates"] >= 5
        assert r["segment_width"] in (L - 1, 2 * L - 2, 3 * L - 3, 4 * L - 4, 6 * L - 6)
        assert r["updates_per_visit"] in (8, 24, 64, 0)
        assert r["phases"] >= 1 and 0 < r["best_ms"] <= r["default_ms"]
        # the tuner left the problem at its starting point: the next solve is a
        # cold start (objective trace starts at E(0)) under the chosen options
        Z = np.zeros((K, Tz), np.float32)
        status, E, st = capi.csc_solve(h, 1e-6, 1 << 40, Z)
        tr = capi.csc_get_trace(h)
        Es = capi.csc_get_objectives(h, len(Xs))
    finally:
        capi.csc_destroy(h)
    assert abs(tr["E_start"] - E0) <= 1e-9 * E0
    assert st["phases"] == r["phases"]
    check_batch(dict(Z=Z, T=T, E=E, Es=Es, stats=st, status=status), D, Xs, lams, refs)


def test_autotune_from_warm_start(capi, short_refs):
    D, Xs, lams, lmax, refs = short_refs
    X, T = batch.pack(Xs)
    L = D.shape[2]
    Z0 = batch.pack_Z([Zr.astype(np.float32) * 0.9 for Zr, _ in refs], L)
    h = capi.csc_setup(cuda(D))
    try:
        capi.csc_init_batch(h, cuda(X), T, lams, cuda(Z0))
        E0 = capi.csc_objective(h, Z0)
        capi.csc_autotune(h, 1e-6)
        Z = np.zeros_like(Z0)
        status, E, st = capi.csc_solve(h, 1e-6, 1 << 40, Z)
        tr = capi.csc_get_trace(h)
        Es = capi.csc_get_objectives(h, len(Xs))
    finally:
        capi.csc_destroy(h)
    assert abs(tr["E_start"] - E0) <= 1e-12 * E0
    check_batch(dict(Z=Z, T=T, E=E, Es=Es, stats=st, status=status), D, Xs, lams, refs)


def test_graph_replay_equals_direct_launches(capi, long_refs):
    # poll batches replayed from a captured CUDA graph (launch indices from
    # device counters) compute exactly what direct launches compute
    D, Xs, lams, refs = long_refs
    a = solve_batch(capi, D, Xs, lams, u=24, launch_mode=0)
    b = solve_batch(capi, D, Xs, lams, u=24, launch_mode=1)
    assert np.array_equal(a["Z"], b["Z"])
    assert a["E"] == b["E"]
    for k in ("updates", "sweeps", "resyncs", "visits"):
        assert a["stats"][k] == b["stats"][k], k
    check_batch(a, D, Xs, lams, refs)


def test_graph_is_captured_once_per_plan(capi, long_refs):
    # the first solve of a plan runs direct launches, the second captures the
    # graph, later ones replay it; every solve computes the same
    D, Xs, lams, refs = long_refs
    X, T = batch.pack(Xs)
    h = capi.csc_setup(cuda(D), capi.make_opts(updates_per_visit=24))
    try:
        launches, Es = [], []
        for _ in range(4):
            capi.csc_init_batch(h, cuda(X), T, lams)
            status, E, st = capi.csc_solve(h, 1e-6)
            assert status == 0
            launches.append(st["kernel_launches"])
            Es.append(E)
    finally:
        capi.csc_destroy(h)
    assert Es[0] == Es[1] == Es[2] == Es[3]
    assert launches[1] == launches[2] == launches[3]
