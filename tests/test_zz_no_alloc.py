"""The allocation-free objective entry point (csc_objective_noalloc).

It serves callers that may not allocate device memory: a serving loop that
admits work against a fixed device-memory budget, or latency-critical code
that cannot take the implicit synchronisation of cudaMalloc/cudaFree.  Its
value must be the objective E(Z) of Eq. sparse_code: the test compares it
with the FP64 oracle's E(Z) (independent of the CUDA path) and with the
handle-based csc_objective on the same D, X, Z and lambda.  Its scratch is a
static device array shared by all calls, so two calls in a row on different
signal lengths check that nothing of the first call leaks into the second.
This file is collected last so that, if it fails, a run that stops at the
first failure has already run every other test.
"""
import ctypes

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


def _case(T, seed):
    pb = synth.make_workload("long_P7_K25_L64_T200000", seed=seed, T=T)
    D = torch.from_numpy(pb.D).cuda()
    X = torch.from_numpy(pb.X).cuda()
    Z = torch.from_numpy(pb.Z_true).cuda()  # any sparse Z: E(Z) is defined for all Z
    return pb, D, X, Z


def _with_handle(capi, D, X, Z, lam):
    h = capi.csc_setup(D)
    try:
        capi.csc_init(h, X, lam)
        return capi.csc_objective(h, Z)
    finally:
        capi.csc_destroy(h)


def test_matches_oracle_and_handle_objective_on_two_calls_in_a_row(capi):
    lam = 0.37
    # first a long signal (many scratch blocks), then a shorter one (fewer)
    for T, seed in ((200_000, 0), (30_001, 5)):
        pb, D, X, Z = _case(T, seed)
        ref = oracle.objective(pb.D, pb.X, pb.Z_true.astype(np.float64), lam)
        want = _with_handle(capi, D, X, Z, lam)
        got = capi.csc_objective_noalloc(D, X, Z, lam)
        # FP64 from the explicit residual on both sides: agreement to 1e-12
        assert got == pytest.approx(ref, rel=1e-12)
        assert got == pytest.approx(want, rel=1e-12)
        dev = torch.zeros(1, dtype=torch.float64, device="cuda")
        got_dev = capi.csc_objective_noalloc(D, X, Z, lam, out=dev)
        assert got_dev == pytest.approx(ref, rel=1e-12)


def test_rejects_signals_beyond_the_static_scratch(capi):
    D = torch.zeros((2, 1, 4), dtype=torch.float32, device="cuda")
    X = torch.zeros((1, 64), dtype=torch.float32, device="cuda")
    Z = torch.zeros((2, 61), dtype=torch.float32, device="cuda")
    lib = capi.load()
    v = ctypes.c_double(0.0)
    st = lib.csc_objective_noalloc(D.data_ptr(), 2, 1, 4, X.data_ptr(), (1 << 24) + 1,
                                   Z.data_ptr(), 0.1, ctypes.addressof(v), None)
    assert st == capi.CSC_EINVAL
    assert "static scratch" in capi.csc_last_error_string()
    # host inputs: refused by the binding, and by the C entry point itself
    with pytest.raises(ValueError):
        capi.csc_objective_noalloc(D.cpu(), X.cpu(), Z.cpu(), 0.1)
    Dh, Xh, Zh = D.cpu(), X.cpu(), Z.cpu()
    st = lib.csc_objective_noalloc(Dh.data_ptr(), 2, 1, 4, Xh.data_ptr(), 64, Zh.data_ptr(),
                                   0.1, ctypes.addressof(v), None)
    assert st == capi.CSC_EINVAL
