"""The seeded input generator: definition, determinism and the recipe of Sec. 4."""
import numpy as np

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
