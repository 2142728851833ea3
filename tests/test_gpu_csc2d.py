"""The 2-D variant on the GPU (csc2d_solve, include/csc2d.h) against the 2-D
FP64 oracle (oracle/csc2d_oracle.c): images cut into row bands (N = 1, the
paper's one-axis cut) or into tiles of row bands x column blocks (N = 0),
run in their phase schedules; the oracle runs the band schedule.  Same bars as the 1-D parity tests: relative objective
gap <= 1e-5, ||Z - Z*||_inf <= 1e-4 ||Z*||_inf, identical support outside
|z| < 1e-6, with Z* the oracle's band-schedule optimum at eps = 1e-10."""
import numpy as np
import pytest

from oracle import csc2d
from paper_1705_10087_gb300 import synth

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


CASES = {
    # K, P, h, w, H, W, rho, sigma, seed, bands
    "small_P2_K3_5x4_40x52": (3, 2, 5, 4, 40, 52, 0.03, 0.05, 3, 4),
    "gray_P1_K8_8x8_128x128": (8, 1, 8, 8, 128, 128, 0.01, 0.1, 5, 8),
    "rgb_P3_K6_6x6_96x80": (6, 3, 6, 6, 96, 80, 0.01, 0.1, 7, 0),
}


def _case(name):
    K, P, h, w, H, W, rho, sigma, seed, M = CASES[name]
    pb = synth.make_problem2d(K=K, P=P, h=h, w=w, H=H, W=W, rho=rho, sigma=sigma, seed=seed)
    lam = 0.1 * csc2d.lambda_max(pb.D, pb.X)
    return pb, lam, M


@pytest.fixture(scope="module")
def refs():
    out = {}
    for name in CASES:
        pb, lam, M = _case(name)
        Hz = pb.X.shape[1] - pb.D.shape[2] + 1
        Mr = M if M else max(1, Hz // (2 * pb.D.shape[2] - 2))
        ref = csc2d.locally_greedy_cd(pb.D, pb.X, lam, 1e-10, M=Mr, mode="phase")
        assert ref["converged"]
        out[name] = (pb, lam, M, ref["Z"], csc2d.objective(pb.D, pb.X, ref["Z"], lam))
    return out


def assert_parity(Z, E, Zr, Er):
    gap = (E - Er) / Er
    assert -1e-9 <= gap <= 1e-5, gap
    assert np.abs(Z - Zr).max() <= 1e-4 * np.abs(Zr).max(), np.abs(Z - Zr).max()
    big = (np.abs(Z) >= 1e-6) | (np.abs(Zr) >= 1e-6)
    assert np.all(np.sign(Z[big]) == np.sign(Zr[big]))


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("u", [0, 3, 1 << 20])
@pytest.mark.parametrize("N", [0, 1, 3])
def test_tile_solve_matches_oracle(capi, refs, name, u, N):
    pb, lam, M, Zr, Er = refs[name]
    K, P, h, w = pb.D.shape
    Hz, Wz = pb.X.shape[1] - h + 1, pb.X.shape[2] - w + 1
    Z = torch.zeros((K, Hz, Wz), dtype=torch.float32, device="cuda")
    status, E, st = capi.csc2d_solve(torch.from_numpy(pb.D).cuda(),
                                     torch.from_numpy(pb.X).cuda(), lam, 1e-6, M=M, N=N,
                                     updates_per_visit=u, Z_out=Z)
    assert status == capi.CSC_OK and st["converged"] == 1, st
    Mo, cr, _ = capi.csc2d_plan(Hz, h, M)
    No, cc, _ = capi.csc2d_plan(Wz, w, N)
    assert (st["bands"], st["col_blocks"], st["phases"]) == (Mo, No, cr * cc)
    assert_parity(Z.cpu().numpy(), E, Zr, Er)
    # the library's objective is E(Z) of the returned Z
    assert E == pytest.approx(csc2d.objective(pb.D, pb.X, Z.cpu().numpy(), lam), rel=1e-10)


def test_host_buffers_and_zero_solution(capi, refs):
    pb, lam, M, Zr, Er = refs["small_P2_K3_5x4_40x52"]
    K, P, h, w = pb.D.shape
    Hz, Wz = pb.X.shape[1] - h + 1, pb.X.shape[2] - w + 1
    Z = np.zeros((K, Hz, Wz), np.float32)
    status, E, st = capi.csc2d_solve(pb.D, pb.X, lam, 1e-6, M=M, Z_out=Z)
    assert status == capi.CSC_OK
    assert_parity(Z, E, Zr, Er)
    # lambda at or above lambda_max: Z* = 0 and E = |X|^2 / 2, no update
    lmax = csc2d.lambda_max(pb.D, pb.X)
    status, E0, st0 = capi.csc2d_solve(pb.D, pb.X, 1.01 * lmax, 1e-6, M=M, Z_out=Z)
    assert status == capi.CSC_OK and st0["updates"] == 0 and not Z.any()
    assert E0 == pytest.approx(0.5 * float((pb.X.astype(np.float64) ** 2).sum()), rel=1e-12)


def test_rejects_bad_arguments(capi):
    D = np.zeros((2, 1, 3, 3), np.float32)
    X = np.zeros((1, 10, 10), np.float32)
    with pytest.raises(capi.CscError):
        capi.csc2d_solve(D, X, -1.0, 1e-6)
    with pytest.raises(capi.CscError):
        capi.csc2d_solve(D, X, 0.1, 1e-6, M=9)  # more bands than rows (Hz = 8)
    with pytest.raises(capi.CscError):
        capi.csc2d_solve(D, X, 0.1, 1e-6, N=9)  # more column blocks than columns
    with pytest.raises(capi.CscError):
        capi.csc2d_solve(D, X, 0.1, 1e-6, N=-1)


def test_dense_refresh_mixes_buckets_and_compaction(capi):
    """A dense optimum (lambda = 0.05 lambda_max): some (row, 32-column tile)
    buckets of Z hold more than their 16 entries, so the exact refresh and the
    objective compact Z per block around those and read the buckets elsewhere.
    Both are checked on the returned Z itself: the reported max |Z - Sh(beta,
    lambda)/n| against the FP64 oracle's beta at that Z (Sec. 2.1), and E
    against the oracle's objective."""
    pb = synth.make_problem2d(K=4, P=1, h=3, w=3, H=30, W=70, rho=0.06, sigma=0.05, seed=11)
    K, P, h, w = pb.D.shape
    Hz, Wz = pb.X.shape[1] - h + 1, pb.X.shape[2] - w + 1
    lam = 0.05 * csc2d.lambda_max(pb.D, pb.X)
    Z = torch.zeros((K, Hz, Wz), dtype=torch.float32, device="cuda")
    status, E, st = capi.csc2d_solve(torch.from_numpy(pb.D).cuda(),
                                     torch.from_numpy(pb.X).cuda(), lam, 1e-6, Z_out=Z)
    assert status in (capi.CSC_OK, capi.CSC_NOT_CONVERGED), st
    Zg = Z.cpu().numpy()
    # both kinds of neighbourhood occur: the refresh block of row i and
    # columns [j0, j0 + 32) reads the buckets of rows i +- (h-1) and of the
    # tiles holding columns [j0 - (w-1), j0 + 32 + w - 1)
    ntc = (Wz + 31) // 32
    cnt = np.array([[np.count_nonzero(Zg[:, i, 32 * t:32 * t + 32]) for t in range(ntc)]
                    for i in range(Hz)])
    over = cnt > 16
    kinds = set()
    for i in range(Hz):
        for t in range(ntc):
            r0, r1 = max(0, i - (h - 1)), min(Hz, i + h)
            c0, c1 = max(0, 32 * t - (w - 1)), min(Wz, 32 * t + 32 + w - 1)
            kinds.add(bool(over[r0:r1, c0 // 32:(c1 - 1) // 32 + 1].any()))
    assert kinds == {True, False}, cnt
    beta = csc2d.beta_fresh(pb.D, pb.X, Zg)
    n = csc2d.norms(pb.D)[:, None, None]
    gap = np.abs(Zg - np.sign(beta) * np.maximum(np.abs(beta) - lam, 0.0) / n).max()
    # the refresh rounds r once to float32 and evaluates the step in float32
    assert abs(st["max_delta_z"] - gap) <= 1e-6 * float((np.abs(beta) / n).max()) + 1e-7, (
        st["max_delta_z"], gap)
    assert E == pytest.approx(csc2d.objective(pb.D, pb.X, Zg, lam), rel=1e-10)
