"""beta0 = D~ * X on the tensor cores (csc_opts.init_mode 1 and 2, and 0 where it
picks them) against the
FP64 oracle, element by element, and a full solve started from it.

Mode 1 splits X and D into three BF16 terms and accumulates six products in
FP32 in tensor memory: its error must be that of an FP32 accumulation, a
multiple of 2^-24 times the sum of |terms| that grows with the number of
16-wide accumulation steps (P * ceil(L/16) of them, each adding the leading
products to the running sum): 4 u per step plus 16 u is the bar.  Mode 2 is
one BF16 product: its error is of BF16 size (about 2^-8 of the sum of |terms|)
and is only measured and bounded here.
"""
import numpy as np
import pytest

import oracle
from paper_1705_10087_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

U = 2.0 ** -24


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


def beta0(capi, pb, mode):
    h = capi.csc_setup(cuda(pb.D), capi.make_opts(init_mode=mode))
    try:
        capi.csc_init(h, cuda(pb.X), 1.0)
        b = torch.zeros((pb.K, pb.Tz), dtype=torch.float32, device="cuda")
        capi.csc_get_beta(h, b)
        lmax = capi.csc_lambda_max(h)
        # a cold-start solve's trace starts at E(0) = sum X^2 / 2 (the kernel's X^2 sum)
        capi.csc_solve(h, 1e30)
        e0 = capi.csc_get_trace(h, 1)["E_start"]
    finally:
        capi.csc_destroy(h)
    return b.cpu().numpy(), lmax, e0


SHAPES = [(5, 1, 16, 2000), (25, 7, 64, 20_000), (3, 2, 5, 5), (25, 1, 200, 3001),
          (1, 1, 1, 700), (64, 7, 64, 3000), (64, 1, 128, 2500), (25, 7, 64, 3 * 128 + 63),
          (33, 2, 20, 1000)]


@pytest.mark.parametrize("K,P,L,T", SHAPES)
def test_tensor_core_beta0_fp32_grade(capi, K, P, L, T):
    pb = synth.make_problem(K=K, P=P, L=L, T=T, rho=0.01, sigma=0.1, seed=2)
    want = oracle.dtx(pb.D, pb.X)
    bound = oracle.dtx(np.abs(pb.D), np.abs(pb.X))
    b, lmax, e0 = beta0(capi, pb, 1)
    err = np.abs(b - want)
    ratio = float((err / np.maximum(bound, 1e-30)).max())
    print(f"mode 1 K={K} P={P} L={L} T={T}: max |err| / sum|terms| = {ratio:.3g} "
          f"= {ratio / U:.2f} u")
    steps = P * ((L + 15) // 16)
    allowed = (4 * steps + 16) * U * bound + 2 * U * np.abs(want)
    assert np.all(err <= allowed), ratio
    assert abs(lmax - np.abs(want).max()) <= allowed.max()
    x2 = float(np.square(pb.X.astype(np.float64)).sum())
    assert e0 == pytest.approx(0.5 * x2, rel=1e-12)


@pytest.mark.parametrize("K,P,L,T", [(25, 7, 64, 20_000), (25, 1, 200, 3001)])
def test_tensor_core_beta0_bf16_error(capi, K, P, L, T):
    pb = synth.make_problem(K=K, P=P, L=L, T=T, rho=0.01, sigma=0.1, seed=2)
    want = oracle.dtx(pb.D, pb.X)
    bound = oracle.dtx(np.abs(pb.D), np.abs(pb.X))
    b, _, _ = beta0(capi, pb, 2)
    ratio = float((np.abs(b - want) / np.maximum(bound, 1e-30)).max())
    print(f"mode 2 K={K} P={P} L={L}: max |err| / sum|terms| = {ratio:.3g}")
    # both operands rounded to 8 significant bits: at most about 2 * 2^-9 per term
    assert ratio <= 2.0 ** -7
    assert ratio >= 2.0 ** -20  # it is a BF16 product, not the FP32 path


def test_solve_from_tensor_core_beta0_parity(capi):
    pb = synth.make_workload("long_P7_K25_L64_T200000", seed=1, T=20_000)
    lam = 0.1 * oracle.lambda_max(pb.D, pb.X)
    ref = oracle.locally_greedy_cd(pb.D, pb.X, lam, 1e-10, M=64, mode="phase")
    Er = oracle.objective(pb.D, pb.X, ref["Z"], lam)
    h = capi.csc_setup(cuda(pb.D), capi.make_opts(init_mode=1, updates_per_visit=24))
    try:
        capi.csc_init(h, cuda(pb.X), lam)
        Z = np.zeros((pb.K, pb.Tz), np.float32)
        status, E, st = capi.csc_solve(h, 1e-6, 1 << 40, Z)
    finally:
        capi.csc_destroy(h)
    assert status == 0
    Eg = oracle.objective(pb.D, pb.X, Z, lam)
    gap = (Eg - Er) / Er
    assert -1e-9 <= gap <= 1e-5
    Zr = ref["Z"]
    assert np.abs(Z - Zr).max() <= 1e-4 * np.abs(Zr).max()
    big = (np.abs(Z) >= 1e-6) | (np.abs(Zr) >= 1e-6)
    assert np.all(np.sign(Z[big]) == np.sign(Zr[big]))


def test_very_long_recording_full_size_sampled(capi):
    """The very long recording (P=1, K=25, L=200, T=5e6) at full size, as the
    default options run it (tensor-core beta0): beta0 on sampled windows
    against the oracle's correlation, the solution's optimality on sampled
    windows from the oracle's fresh FP64 beta (which needs Z only within L-1
    of the window), and the library's objective against the oracle's."""
    pb = synth.make_workload("verylong_P1_K25_L200_T5000000", seed=0)
    K, L, Tz = pb.K, pb.L, pb.Tz
    D, X = cuda(pb.D), cuda(pb.X)
    h = capi.csc_setup(D, capi.make_opts(updates_per_visit=24))
    try:
        capi.csc_init(h, X, 1.0)
        lam = 0.1 * capi.csc_lambda_max(h)
        capi.csc_init(h, X, lam)
        b0 = torch.zeros((K, Tz), dtype=torch.float32, device="cuda")
        capi.csc_get_beta(h, b0)
        Zd = torch.zeros((K, Tz), dtype=torch.float32, device="cuda")
        status, E, st = capi.csc_solve(h, 1e-6, 1 << 40, Zd)
    finally:
        capi.csc_destroy(h)
    assert status == 0 and st["converged"] == 1
    b0 = b0.cpu().numpy()
    Z = Zd.cpu().numpy()
    n = oracle.norms(pb.D)
    steps = pb.P * ((L + 15) // 16)
    for a in (0, 1_234_567, 3_000_001, Tz - 1000):
        b = min(a + 1000, Tz)
        want = oracle.dtx(pb.D, pb.X[:, a:b + L - 1])
        bound = oracle.dtx(np.abs(pb.D), np.abs(pb.X[:, a:b + L - 1]))
        err = np.abs(b0[:, a:b] - want)
        allowed = (4 * steps + 16) * U * bound + 2 * U * np.abs(want)
        assert np.all(err <= allowed)
        # fresh beta on the window [a, b): Z on [a-L+1, b+L-1), X on [a-L+1, b+2L-2)
        lo = max(0, a - L + 1)
        zw = Z[:, lo:min(Tz, b + L - 1)]
        xw = pb.X[:, lo:min(pb.T, lo + zw.shape[1] + L - 1)]
        beta_w = oracle.beta_fresh(pb.D, xw, zw)[:, a - lo:b - lo]
        k = oracle.kkt(beta_w, Z[:, a:b], n, lam)
        # the solve is optimal for its own beta0: against the exact problem the
        # coordinate gaps may also carry beta0's error (divided by ||D_k||^2 = 1)
        slack = float(allowed.max())
        assert k["zero_excess"] <= 1e-6 * lam + slack, k
        assert k["max_delta_z"] <= 2e-6 + slack, k
    Eo = oracle.objective(pb.D, pb.X, Z, lam)
    assert abs(E - Eo) <= 1e-9 * Eo


def test_very_long_recording_full_size_parity(capi):
    """The very long recording at full size (K x Tz = 25 x 4,999,801 coordinates)
    with the default options (tensor-core beta0, automatic segments) against
    the oracle's optimum stored by tests/golden/make_golden.py --verylong
    (phase-schedule locally greedy CD at eps = 1e-10): relative objective gap
    <= 1e-5, ||Z - Z*||_inf <= 1e-4 ||Z*||_inf and the same support outside
    |z| < 1e-6, over every coordinate (compared on the device)."""
    import hashlib
    import json
    import os
    gdir = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
    name = "verylong_P1_K25_L200_T5000000"
    with open(os.path.join(gdir, "optimum.json")) as f:
        g = json.load(f)[f"{name}/seed0"]
    pb = synth.make_workload(name, seed=0)
    hsh = hashlib.sha256()
    hsh.update(pb.D.tobytes())
    hsh.update(pb.X.tobytes())
    assert hsh.hexdigest()[:16] == g["input_sha256_16"], "generator drifted from the stored inputs"
    zs = np.load(os.path.join(gdir, g["zstar"]))
    K, Tz = pb.K, pb.Tz
    assert tuple(zs["shape"]) == (K, Tz)
    lam = g["lambda"]
    h = capi.csc_setup(cuda(pb.D), capi.make_opts(updates_per_visit=24))
    try:
        capi.csc_init(h, cuda(pb.X), lam)
        Zd = torch.zeros((K, Tz), dtype=torch.float32, device="cuda")
        status, E, st = capi.csc_solve(h, 1e-6, 1 << 40, Zd)
    finally:
        capi.csc_destroy(h)
    assert status == 0 and st["converged"] == 1, st
    gap = (E - g["E_star"]) / g["E_star"]
    assert -1e-9 <= gap <= 1e-5, gap
    idx = torch.from_numpy(zs["index"]).cuda()
    zstar = torch.zeros(K * Tz, dtype=torch.float32, device="cuda")
    zstar[idx] = torch.from_numpy(zs["value"]).cuda()
    zg = Zd.view(-1)
    zinf = float(zstar.abs().max())
    assert zinf == pytest.approx(g["zinf"], rel=1e-6)
    assert float((zg - zstar).abs().max()) <= 1e-4 * zinf
    big = (zg.abs() >= 1e-6) | (zstar.abs() >= 1e-6)
    mismatched = int((torch.sign(zg[big]) != torch.sign(zstar[big])).sum())
    assert mismatched == 0, mismatched
