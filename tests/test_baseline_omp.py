"""The multi-core CPU baseline (oracle/csc_baseline_omp.c) runs the segments
of a phase on several threads; because co-active segments never touch the
same beta entries, it must reproduce the single-threaded oracle's phase
schedule exactly (same updates, bit-identical Z) for every thread count."""
import numpy as np
import pytest

import oracle
from oracle import baseline_omp
from paper_1705_10087_gb300 import synth


@pytest.mark.parametrize("name,T,M,u", [("short_P1_K5_L16_T2000", None, 10, 0),
                                        ("long_P7_K25_L64_T200000", 6000, 24, 24),
                                        ("long_P7_K25_L64_T200000", 6000, 70, 3)])
def test_matches_oracle_phase_schedule_bitwise(name, T, M, u):
    pb = synth.make_workload(name, seed=2, T=T)
    lam = 0.1 * oracle.lambda_max(pb.D, pb.X)
    ref = oracle.locally_greedy_cd(pb.D, pb.X, lam, 1e-9, M=M, mode="phase",
                                   updates_per_visit=u)
    for threads in (1, 4):
        got = baseline_omp.phase_cd(pb.D, pb.X, lam, 1e-9, M, u, threads=threads)
        assert got["converged"] and ref["converged"]
        assert got["n_updates"] == ref["n_updates"]
        assert np.array_equal(got["Z"], ref["Z"])
