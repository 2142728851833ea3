"""The multi-process solve of one signal (include/csc_shard.h,
paper_1705_10087_gb300/shard.py) on CPU: the host-only partition plan against
the single-process segment schedule, and the exchange protocol run by gloo
ranks over a float64 numpy stand-in for each rank's GPU calls.  The sharded
run must perform the single-process run's updates (the same count, the same
Z up to the order of border additions) and reach the oracle's optimum."""
import os
import socket
import sys

import numpy as np
import pytest

import oracle
from paper_1705_10087_gb300 import build, capi, shard, synth

torch = pytest.importorskip("torch")
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    build.build()
    return capi.load()


PLANS = [(2000, 16, 10, 2), (2000, 16, 10, 3), (20_000, 64, 64, 4), (20_000, 64, 100, 7),
         (5000, 1, 50, 5), (200_000, 64, 1024, 8), (5_000_000, 200, 12_562, 8), (300, 8, 12, 4)]


@pytest.mark.parametrize("T,L,M,world", PLANS)
def test_plan_partitions_the_single_process_schedule(lib, T, L, M, world):
    Tz = T - L + 1
    plans = [capi.csc_shard_plan_make(T, L, M, world, q) for q in range(world)]
    c = oracle.phase_count(Tz, M, L)
    seg, col = 0, 0
    for q, p in enumerate(plans):
        assert (p["T"], p["Tz"], p["L"], p["M"], p["world"], p["rank"]) == (T, Tz, L, M, world, q)
        assert p["phases"] == c
        # contiguous runs of the single-process segments, in rank order
        assert p["seg_first"] == seg and p["seg_count"] >= 1
        assert p["col_first"] == oracle.segment_start(Tz, M, seg) == col
        seg += p["seg_count"]
        assert p["col_first"] + p["col_count"] == oracle.segment_start(Tz, M, seg)
        col += p["col_count"]
        # halos: L-1 columns on each side that has a neighbour
        assert p["halo_left"] == (min(L - 1, p["col_first"]) if q > 0 else 0)
        assert p["halo_right"] == (min(L - 1, Tz - col) if q < world - 1 else 0)
        assert p["col_count"] >= L - 1
        assert p["x_first"] == p["col_first"] - p["halo_left"]
        assert p["x_count"] == p["col_count"] + p["halo_left"] + p["halo_right"] + L - 1
        if q > 0:  # my left halo is exactly my left neighbour's right halo's width
            assert p["halo_left"] == plans[q - 1]["halo_right"]
    assert seg == M and col == Tz


def test_plan_rejects_bad_requests(lib):
    with pytest.raises(capi.CscError):
        capi.csc_shard_plan_make(2000, 16, 10, 11, 0)  # more ranks than segments
    with pytest.raises(capi.CscError):
        capi.csc_shard_plan_make(100, 64, 4, 4, 0)  # shards narrower than L-1
    with pytest.raises(capi.CscError):
        capi.csc_shard_plan_make(2000, 16, 10, 2, 2)  # rank out of range


def _problem():
    # seed 1: the optimum has activations within L-1 on both sides of every
    # border of the 2- and 3-rank plans, so the halos carry changes
    pb = synth.make_problem(K=3, P=2, L=8, T=420, rho=0.06, sigma=0.1, seed=1)
    lam = 0.1 * oracle.lambda_max(pb.D, pb.X)
    return pb, lam


M_SEG, U = 24, 3


def _run_rank(rank, world, comm, make):
    sys.path.insert(0, os.path.join(ROOT, "tests"))
    from shard_np import NumpyShard
    pb, lam = _problem()
    plan = capi.csc_shard_plan_make(pb.T, pb.L, M_SEG, world, rank)
    Xw = pb.X[:, plan["x_first"]:plan["x_first"] + plan["x_count"]]
    be = NumpyShard(pb.D, Xw, plan, lam, u=U)
    res = shard.solve(be, comm, pb.K, plan, tol=1e-11, make=make)
    res["sent"] = be.sent
    return plan, be.get_z(), res


def _worker(rank, world, port, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank,
                            world_size=world)
    try:
        comm = shard.TorchComm(dist)
        plan, Z, res = _run_rank(rank, world, comm,
                                 lambda shape: torch.zeros(shape, dtype=torch.float64))
        out[rank] = (plan["col_first"], Z, res)
        dist.barrier()
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_sharded_protocol_gloo(lib, world):
    sys.path.insert(0, os.path.join(ROOT, "tests"))
    from shard_np import LocalComm
    import torch.multiprocessing as mp
    with socket.socket() as sk:
        sk.bind(("127.0.0.1", 0))
        port = sk.getsockname()[1]
    out = mp.Manager().dict()
    mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
    parts = [out[q] for q in range(world)]
    Z = np.concatenate([p[1] for p in parts], axis=1)
    # one rank, same stand-in, same schedule
    _, Z1, res1 = _run_rank(0, 1, LocalComm(), lambda shape: np.zeros(shape))
    for _, _, res in parts:
        assert res["converged"] and res1["converged"]
        assert res["updates"] == res1["updates"]  # the same updates ...
        assert res["E"] == pytest.approx(res1["E"], rel=1e-12)
    assert np.abs(Z - Z1).max() <= 1e-12 * np.abs(Z1).max()  # ... up to border order
    # updates near every border: the neighbours' changes did travel
    assert all(p[2]["sent"] > 0 for p in parts)
    # and the optimum of the problem
    pb, lam = _problem()
    ref = oracle.greedy_cd(pb.D, pb.X, lam, 1e-12)
    assert np.abs(Z - ref["Z"]).max() <= 1e-8 * np.abs(ref["Z"]).max()
    Er = oracle.objective(pb.D, pb.X, ref["Z"], lam)
    assert parts[0][2]["E"] == pytest.approx(Er, rel=1e-12)


def test_numpy_stand_in_single_rank_reaches_the_oracle(lib):
    sys.path.insert(0, os.path.join(ROOT, "tests"))
    from shard_np import LocalComm
    pb, lam = _problem()
    _, Z, res = _run_rank(0, 1, LocalComm(), lambda shape: np.zeros(shape))
    ref = oracle.locally_greedy_cd(pb.D, pb.X, lam, 1e-12, M=M_SEG, mode="phase",
                                   updates_per_visit=U)
    assert res["converged"]
    assert np.abs(Z - ref["Z"]).max() <= 1e-9 * np.abs(ref["Z"]).max()
