"""Failure detection without a GPU fault.

Every device-side wait of the library is a bounded poll (the tensor-core beta0
kernel's mbarrier waits).  csc_check_wait_timeout runs that wait on an mbarrier
that nothing arrives at: the wait must give up within its poll limit, the
kernel must return, the call must report CSC_ETIMEOUT, and the device must
stay usable (a solve right after it still matches the FP64 oracle).  Nothing
here traps, faults or hangs the GPU: the wait ends after a fixed number of
polls.
"""
import time

import numpy as np
import pytest

import oracle
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


@pytest.mark.parametrize("polls", [1, 4096])
def test_bounded_wait_gives_up_and_device_stays_usable(capi, polls):
    t0 = time.perf_counter()
    st = capi.csc_check_wait_timeout(polls)
    dt = time.perf_counter() - t0
    assert st == capi.CSC_ETIMEOUT, capi.csc_last_error_string()
    assert "gave up" in capi.csc_last_error_string()
    assert dt < 10.0
    # the context is intact: a small solve right after still matches the oracle
    pb = synth.make_problem(K=5, P=2, L=16, T=1500, rho=0.01, sigma=0.1, seed=31)
    lam = 0.1 * oracle.lambda_max(pb.D, pb.X)
    ref = oracle.locally_greedy_cd(pb.D, pb.X, lam, 1e-10, M=8, mode="phase")
    Er = oracle.objective(pb.D, pb.X, ref["Z"], lam)
    D = torch.from_numpy(pb.D).cuda()
    X = torch.from_numpy(pb.X).cuda()
    h = capi.csc_setup(D, capi.make_opts(init_mode=1))
    try:
        capi.csc_init(h, X, lam)
        Z = np.zeros((pb.K, pb.Tz), np.float32)
        status, E, _ = capi.csc_solve(h, 1e-6, 1 << 40, Z)
    finally:
        capi.csc_destroy(h)
    assert status == 0
    Eg = oracle.objective(pb.D, pb.X, Z, lam)
    assert -1e-9 <= (Eg - Er) / Er <= 1e-5
    torch.cuda.synchronize()
