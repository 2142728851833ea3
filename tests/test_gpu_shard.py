"""The multi-process solve of one signal through the C ABI (include/csc_shard.h)
on one GPU: two processes, each with its own handle on cuda:0, own contiguous
runs of segments of one signal and exchange their halos through gloo on host
buffers between phases (no kernel of one process waits for the other).  The
assembled Z must meet the parity bars against the FP64 oracle's optimum."""
import os
import socket
import sys

import numpy as np
import pytest

import oracle
from paper_1705_10087_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

WORKLOAD, SEED, T, M = "long_P7_K25_L64_T200000", 1, 20_000, 64


def _worker(rank, world, port, tol, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    from paper_1705_10087_gb300 import build, capi, shard
    torch.cuda.set_device(0)
    build.build()
    capi.load()
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank,
                            world_size=world)
    try:
        pb = synth.make_workload(WORKLOAD, seed=SEED, T=T)
        lam = 0.1 * oracle.lambda_max(pb.D, pb.X)
        plan = capi.csc_shard_plan_make(pb.T, pb.L, M, world, rank)
        Xw = np.ascontiguousarray(pb.X[:, plan["x_first"]:plan["x_first"] + plan["x_count"]])
        h = capi.csc_setup(torch.from_numpy(pb.D).cuda(), capi.make_opts(updates_per_visit=24))
        try:
            capi.csc_shard_init(h, plan, torch.from_numpy(Xw).cuda(), lam)
            be = shard.CapiShard(capi, h, plan)
            res = shard.solve(be, shard.TorchComm(dist), pb.K, plan, tol,
                              make=lambda shape: torch.zeros(shape, dtype=torch.float32))
            Z = torch.zeros((pb.K, plan["col_count"]), dtype=torch.float32, device="cuda")
            be.get_z(Z)
            out[rank] = (Z.cpu().numpy(), res)
        finally:
            capi.csc_destroy(h)
        dist.barrier()
    finally:
        dist.destroy_process_group()


@pytest.fixture(scope="module")
def reference():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    pb = synth.make_workload(WORKLOAD, seed=SEED, T=T)
    lam = 0.1 * oracle.lambda_max(pb.D, pb.X)
    ref = oracle.locally_greedy_cd(pb.D, pb.X, lam, 1e-10, M=M, mode="phase")
    assert ref["converged"]
    return pb, lam, ref["Z"], oracle.objective(pb.D, pb.X, ref["Z"], lam)


@pytest.mark.parametrize("world", [2])
def test_two_processes_one_signal_parity(reference, world):
    import torch.multiprocessing as mp
    pb, lam, Zr, Er = reference
    with socket.socket() as sk:
        sk.bind(("127.0.0.1", 0))
        port = sk.getsockname()[1]
    out = mp.Manager().dict()
    mp.spawn(_worker, args=(world, port, 1e-6, out), nprocs=world, join=True)
    parts = [out[q] for q in range(world)]
    Z = np.concatenate([p[0] for p in parts], axis=1)
    assert Z.shape == Zr.shape
    for _, res in parts:
        assert res["converged"], res
    E = parts[0][1]["E"]
    assert all(p[1]["E"] == E for p in parts)  # one reduced value on every rank
    gap = (E - Er) / Er
    assert -1e-9 <= gap <= 1e-5, gap
    assert np.abs(Z - Zr).max() <= 1e-4 * np.abs(Zr).max()
    big = (np.abs(Z) >= 1e-6) | (np.abs(Zr) >= 1e-6)
    assert np.all(np.sign(Z[big]) == np.sign(Zr[big]))
    # the objective summed over ranks is the objective of the assembled Z
    assert E == pytest.approx(oracle.objective(pb.D, pb.X, Z, lam), rel=1e-9)
