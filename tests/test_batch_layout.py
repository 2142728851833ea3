"""Host-side layout of batches (no GPU): packing, offsets, straddling columns,
and the batch workload's length distribution."""
import numpy as np
import pytest

from paper_1705_10087_gb300 import batch, synth


def test_pack_and_unpack_round_trip():
    rng = np.random.default_rng(0)
    L, K = 5, 3
    Ts = [5, 9, 40, 6]
    Xs = [rng.standard_normal((2, T)).astype(np.float32) for T in Ts]
    X, T = batch.pack(Xs)
    assert X.shape == (2, sum(Ts)) and list(T) == Ts
    a = batch.offsets(T)
    assert list(a) == [0, 5, 14, 54, 60]
    for i, x in enumerate(Xs):
        assert np.array_equal(X[:, a[i]:a[i + 1]], x)
    Zs = [rng.standard_normal((K, t - L + 1)).astype(np.float32) for t in Ts]
    Z = batch.pack_Z(Zs, L)
    assert Z.shape == (K, sum(Ts) - L + 1)
    for z, zz in zip(Zs, batch.unpack_Z(Z, T, L)):
        assert np.array_equal(z, zz)
    m = batch.straddle_mask(T, L)
    # L - 1 straddling columns after every signal but the last
    assert m.sum() == (L - 1) * (len(Ts) - 1)
    assert not np.any(Z[:, m])
    # a valid column of signal i and one of signal i+1 are at least L apart
    for i in range(len(Ts) - 1):
        assert (a[i + 1]) - (a[i + 1] - L) == L


def test_pack_rejects_mismatched_channels():
    with pytest.raises(ValueError):
        batch.pack([np.zeros((2, 10), np.float32), np.zeros((3, 10), np.float32)])
    with pytest.raises(ValueError):
        batch.pack([])


def test_batch_lengths_distribution():
    T = synth.batch_lengths(4096, 10_000, 500_000, seed=0)
    assert T.min() >= 10_000 and T.max() <= 500_000
    # uniform: mean (a+b)/2 within 4 standard errors
    sd = (500_000 - 10_000) / np.sqrt(12) / np.sqrt(T.size)
    assert abs(T.mean() - 255_000) < 4 * sd
    assert np.array_equal(T, synth.batch_lengths(4096, 10_000, 500_000, seed=0))


def test_make_batch_shares_dictionary():
    pbs = synth.make_batch("batch_P7_K25_L64_n512_T10000_500000", seed=0, n=3, T_max=2000)
    assert len(pbs) == 3
    for pb in pbs:
        assert np.array_equal(pb.D, pbs[0].D)
        assert pb.X.shape[0] == 7 and 2000 >= pb.T >= 64
    assert not np.array_equal(pbs[0].Z_true[:, :100], pbs[1].Z_true[:, :100])
