"""The seeded input generator: definition, determinism and the recipe of Sec. 4."""
import numpy as np
import pytest

from paper_1705_10087_gb300 import synth
from tests import npref


def test_splitmix64_reference_outputs():
    # first two outputs of SplitMix64 from state 0 (Steele, Lea & Flood 2014)
    with np.errstate(over="ignore"):
        x = np.array([synth._GOLDEN, synth._GOLDEN * np.uint64(2)], dtype=np.uint64)
    got = [int(v) for v in synth._mix64(x)]
    assert got == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4]


def test_deterministic_and_seed_dependent():
    a = synth.make_problem(K=3, P=2, L=8, T=500, rho=0.05, sigma=0.1, seed=4)
    b = synth.make_problem(K=3, P=2, L=8, T=500, rho=0.05, sigma=0.1, seed=4)
    c = synth.make_problem(K=3, P=2, L=8, T=500, rho=0.05, sigma=0.1, seed=5)
    for f in ("D", "Z_true", "X"):
        np.testing.assert_array_equal(getattr(a, f), getattr(b, f))
        assert not np.array_equal(getattr(a, f), getattr(c, f))


def test_distributions():
    u = synth.uniform(0, 1, 200_000)
    assert u.min() > 0 and u.max() < 1 and abs(u.mean() - 0.5) < 0.005
    g = synth.normal(0, 2, 200_000)
    assert abs(g.mean()) < 0.01 and abs(g.std() - 1) < 0.01


def test_recipe_of_the_long_signal_workload():
    # unit-norm Gaussian atoms, Bernoulli(rho)-Gaussian Z, X = sum Z*D + sigma noise
    pb = synth.make_workload("long_P7_K25_L64_T200000", seed=0, T=20_000)
    assert pb.D.shape == (25, 7, 64) and pb.X.shape == (7, 20_000) and pb.D.dtype == np.float32
    np.testing.assert_allclose((pb.D.astype(np.float64) ** 2).sum(axis=(1, 2)), 1.0, rtol=1e-6)
    dens = np.count_nonzero(pb.Z_true) / pb.Z_true.size
    assert abs(dens - 0.005) < 0.0008
    noise = npref.residual(pb.D, pb.X, pb.Z_true.astype(np.float64))
    assert abs(noise.std() - 0.1) < 0.003


def test_indexed_draws_equal_full_draws():
    idx = np.array([0, 5, 17, 999, 3])
    assert np.array_equal(synth.uniform_at(4, 7, idx), synth.uniform(4, 7, 1000)[idx])
    assert np.array_equal(synth.normal_at(4, 7, idx), synth.normal(4, 7, 1000)[idx])


def test_bernoulli_support_law():
    # n Bernoulli(rho) trials drawn as geometric gaps: the count is Binomial(n, rho)
    # and every index is hit with probability rho, whatever its position
    n, rho = 2_000_000, 0.005
    s = synth.bernoulli_support(11, 3, n, rho)
    assert np.all(np.diff(s) > 0) and s[0] >= 0 and s[-1] < n
    sd = np.sqrt(n * rho * (1 - rho))
    assert abs(s.size - n * rho) < 5 * sd
    # rate in the first and last tenth agree with rho (no drift along the signal)
    for lo in (0, 9 * n // 10):
        c = np.count_nonzero((s >= lo) & (s < lo + n // 10))
        assert abs(c - n * rho / 10) < 5 * np.sqrt(n / 10 * rho)
    # P(gap > g) = (1 - rho)^g: gaps beyond the median of the geometric law
    g = np.diff(s)
    med = np.log(0.5) / np.log1p(-rho)
    assert abs(np.mean(g > med) - 0.5) < 5 * 0.5 / np.sqrt(g.size)
    # edge cases
    assert synth.bernoulli_support(1, 3, 0, 0.5).size == 0
    assert synth.bernoulli_support(1, 3, 10, 0.0).size == 0
    assert np.array_equal(synth.bernoulli_support(1, 3, 10, 1.0), np.arange(10))
    assert np.array_equal(s, synth.bernoulli_support(11, 3, n, rho))


def test_gaps_support_problem():
    pb = synth.make_problem(K=5, P=2, L=8, T=50_000, rho=0.01, sigma=0.1, seed=3,
                            support="gaps")
    nz = np.count_nonzero(pb.Z_true)
    N = 5 * (50_000 - 7)
    assert abs(nz - 0.01 * N) < 5 * np.sqrt(0.01 * N)
    amp = pb.Z_true[pb.Z_true != 0]
    assert abs(amp.std() - 1.0) < 0.05 and abs(amp.mean()) < 0.05


def test_request_stream_schedule_law():
    # Poisson arrivals at 200 req/s (exponential gaps: mean 1/rate, CV 1),
    # dictionary uniform over four, length log-uniform on [5e3, 2e6]
    name = "serve_4dict_poisson200_T5000_2000000"
    n = 40_000
    s = synth.serve_schedule(name, n, seed=0)
    gaps = np.diff(np.concatenate([[0.0], s["arrival"]]))
    assert np.all(gaps > 0)
    assert gaps.mean() == pytest.approx(1 / 200, rel=0.02)
    assert gaps.std() / gaps.mean() == pytest.approx(1.0, abs=0.03)
    counts = np.bincount(s["dict"], minlength=4)
    assert counts.shape == (4,) and np.all(np.abs(counts / n - 0.25) < 0.01)
    assert s["T"].min() >= 5_000 and s["T"].max() <= 2_000_000
    u = (np.log(s["T"]) - np.log(5_000)) / (np.log(2_000_000) - np.log(5_000))
    assert u.mean() == pytest.approx(0.5, abs=0.01)
    assert np.median(s["T"]) == pytest.approx(1e5, rel=0.05)
    assert np.all((s["offset_frac"] >= 0) & (s["offset_frac"] < 1))
    # the same seed gives the same stream; a shorter prefix is a prefix
    s2 = synth.serve_schedule(name, 100, seed=0)
    assert np.array_equal(s2["arrival"], s["arrival"][:100])
    assert np.array_equal(s2["T"], s["T"][:100])
    # T_max caps lengths without changing arrivals or dictionaries
    s3 = synth.serve_schedule(name, 100, seed=0, T_max=20_000)
    assert s3["T"].max() <= 20_000 and np.array_equal(s3["dict"], s2["dict"])


def test_stream_sources_same_with_worker_processes():
    # one recording per dictionary, (K, L, P) as the stream names them; the
    # spawned worker pool yields exactly the serial result
    name = "serve_4dict_poisson200_T5000_2000000"
    a = synth.serve_sources(name, seed=1, T_source=3000)
    b = synth.serve_sources(name, seed=1, T_source=3000, workers=2)
    assert [(pb.K, pb.L, pb.P) for pb in a] == [tuple(d) for d in
                                               synth.SERVE_WORKLOADS[name]["dicts"]]
    for x, y in zip(a, b):
        assert np.array_equal(x.D, y.D) and np.array_equal(x.X, y.X)
        assert x.X.shape == (x.P, 3000)
        # unit-norm atoms (Sec. 4 recipe)
        assert np.allclose(np.sqrt((x.D.astype(np.float64) ** 2).sum(axis=(1, 2))), 1.0,
                           atol=1e-6)


def test_image_problem_recipe():
    # unit-norm atoms, Bernoulli(rho) support, and X minus the model is the
    # noise: the 2-D oracle's residual at Z_true has the noise's spread
    from oracle import csc2d
    pb = synth.make_problem2d(K=4, P=2, h=5, w=4, H=60, W=50, rho=0.01, sigma=0.1, seed=3)
    assert pb.D.dtype == np.float32 and pb.X.shape == (2, 60, 50)
    assert np.allclose(np.sqrt((pb.D.astype(np.float64) ** 2).sum(axis=(1, 2, 3))), 1.0,
                       atol=1e-6)
    assert pb.Z_true.shape == (4, 56, 47)
    dens = np.count_nonzero(pb.Z_true) / pb.Z_true.size
    assert 0.005 < dens < 0.02
    R = csc2d.residual(pb.D, pb.X, pb.Z_true)
    assert R.std() == pytest.approx(0.1, rel=0.05) and abs(R.mean()) < 0.01
    again = synth.make_problem2d(K=4, P=2, h=5, w=4, H=60, W=50, rho=0.01, sigma=0.1, seed=3)
    assert np.array_equal(again.X, pb.X) and np.array_equal(again.Z_true, pb.Z_true)
