"""The multi-rank path of bench.py on CPU (gloo, world size 2): N replicas
solve independent seeds with no collective on the data path; the job's time is
the slowest rank's and its units the sum over ranks; the reference arm runs on
rank 0 only."""
import os
import sys

import pytest

torch = pytest.importorskip("torch")
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _worker(rank, world, port, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank,
                            world_size=world)
    try:
        # rank r: its own elapsed time and units (as if it solved seed r)
        elapsed, units = 10.0 + 5.0 * rank, 1000 * (rank + 1)
        t, u = bench.over_ranks(dist, "cpu", elapsed, units)
        dist.barrier()
        out[rank] = (t, u)
    finally:
        dist.destroy_process_group()


def test_over_ranks_gloo_world_two():
    import socket
    import torch.multiprocessing as mp
    with socket.socket() as sk:
        sk.bind(("127.0.0.1", 0))
        port = sk.getsockname()[1]
    out = mp.Manager().dict()
    mp.spawn(_worker, args=(2, port, out), nprocs=2, join=True)
    # every rank sees the max time and the summed units
    assert out[0] == (15.0, 3000.0) and out[1] == (15.0, 3000.0)


def test_over_ranks_single_process():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.over_ranks(None, "cpu", 12.5, 7) == (12.5, 7.0)


def test_reference_arm_runs_on_rank_zero_only(monkeypatch):
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setenv("RANK", "1")
    # a non-zero rank returns before touching the oracle or the generator
    class A:
        warmup, steps, tol, segments, updates_per_visit, gpus = 1, 1, 1e-6, 1024, 24, 2
    assert bench.run_reference(A()) is None


def test_replicas_solve_distinct_seeds():
    # rank r solves seed r: different inputs, same workload shape (weak scaling)
    sys.path.insert(0, ROOT)
    from paper_1705_10087_gb300 import synth
    a = synth.make_workload("short_P1_K5_L16_T2000", seed=0)
    b = synth.make_workload("short_P1_K5_L16_T2000", seed=1)
    assert a.X.shape == b.X.shape and not (a.X == b.X).all()


def test_time_to_gap_from_the_objective_trace():
    # E after each launch = E_start - cumulative decrease; the first launch at
    # which (E - E*) <= 1e-4 E* gives the time, from the last time stamp up to it
    sys.path.insert(0, ROOT)
    import numpy as np
    import bench
    tr = {"E_start": 10.0, "decrease": np.array([5.0, 3.0, 0.99995, 0.0, 1e-5]),
          "t_ns": np.array([1_000_000, 2_000_000, 3_000_000, -1, 5_000_000])}
    assert bench.time_to_gap_ms(tr, 0.5, 1.0) == pytest.approx(3.5)
    # reached at a launch without a time stamp: the last stamped launch before it
    tr2 = dict(tr, t_ns=np.array([1_000_000, 2_000_000, -1, -1, 5_000_000]))
    assert bench.time_to_gap_ms(tr2, 0.0, 1.0) == pytest.approx(2.0)
    # never within the gap
    assert bench.time_to_gap_ms(tr, 0.5, 1.0, rel=1e-6) is None
