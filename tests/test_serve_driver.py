"""The stream driver's host loop (serve.run_stream) against a fake server, on
CPU: requests are submitted in arrival order and not before their arrival
time, every finished request is reported once by the completion queue and
fetched once into a buffer of its own shape, and the reported counters come
from the server.  The fake stands in for libcsc's csc_server_* calls; the
solver itself is covered by tests/test_gpu_server.py."""
import time
import types

import numpy as np
import pytest

from paper_1705_10087_gb300 import serve, synth

torch = pytest.importorskip("torch")


class _Pinnable:
    def __init__(self, t):
        self.t = t

    def pin_memory(self):
        return self.t


class FakeTorch:
    float32 = torch.float32

    @staticmethod
    def empty(n, dtype):
        return _Pinnable(torch.empty(n, dtype=dtype))


class FakeServer:
    """Each request finishes after a fixed number of scheduling rounds."""
    CSC_REQ_DONE = 2

    def __init__(self, rounds=3):
        self.rounds = rounds
        self.dicts, self.widths, self.reqs, self.queue = [], [], {}, []
        self.submitted, self.fetched = [], []
        self.next_id, self.launches, self.destroyed = 1, 0, False
        self.t_first_count = None  # the driver reads the counter just before its clock starts

    def csc_server_create(self, hbm_budget_bytes, sweeps_per_step):
        assert hbm_budget_bytes > 0
        return "srv"

    def csc_server_add_dictionary(self, srv, D, segment_width=0):
        assert segment_width >= 0
        self.dicts.append(D.shape)
        self.widths.append(segment_width)
        return len(self.dicts) - 1

    def csc_server_submit(self, srv, d, X, lam, tol):
        assert lam < 0 and tol > 0  # relative lambda, positive tolerance
        K, P, L = self.dicts[d]
        assert X.shape[0] == P and X.flags.c_contiguous
        rid = self.next_id
        self.next_id += 1
        self.reqs[rid] = dict(K=K, L=L, T=X.shape[1], left=self.rounds, done=False)
        self.submitted.append((rid, time.perf_counter()))
        return rid

    def csc_server_step(self, srv):
        self.launches += 1
        for rid, q in self.reqs.items():
            if not q["done"]:
                q["left"] -= 1
                if q["left"] == 0:
                    q["done"] = True
                    self.queue.append(rid)
        active = sum(1 for q in self.reqs.values() if not q["done"])
        return active, 0, len(self.reqs) - active

    def csc_server_completed(self, srv):
        out, self.queue = self.queue, []
        return out

    def csc_server_fetch(self, srv, rid, Z):
        q = self.reqs.pop(rid)  # released: a second fetch would fail
        assert q["done"]
        assert tuple(Z.shape) == (q["K"], q["T"] - q["L"] + 1)
        Z.fill_(float(rid))
        self.fetched.append(rid)
        return {"converged": 1}

    def csc_server_kernel_launches(self, srv):
        if self.t_first_count is None:
            self.t_first_count = time.perf_counter()
        return self.launches

    def csc_server_memory(self, srv):
        return {"peak": 123, "pool_bytes": 456}

    def csc_server_destroy(self, srv):
        self.destroyed = True


def sources(T):
    w = synth.SERVE_WORKLOADS[serve.WORKLOAD]
    rng = np.random.default_rng(0)
    return [types.SimpleNamespace(D=np.zeros((K, P, L), np.float32), K=K, L=L, T=T,
                                  X=rng.standard_normal((P, T)).astype(np.float32))
            for K, L, P in w["dicts"]]


def test_stream_driver_submits_on_time_and_fetches_each_request_once():
    n, rate, T = 40, 2000.0, 600
    fake = FakeServer(rounds=3)
    out = serve.run_stream(fake, FakeTorch, n, seed=0, rate=rate, sources=sources(2 * T),
                           T_max=T, keep_Z=True)
    sch = out["schedule"]
    ids = [rid for rid, _ in fake.submitted]
    assert ids == list(range(1, n + 1))                      # arrival order
    assert sorted(fake.fetched) == ids                       # each fetched once
    assert fake.destroyed and not fake.reqs
    # not before its arrival: the clock starts after the first counter read
    ts = np.array([t for _, t in fake.submitted])
    assert np.all(ts - fake.t_first_count >= sch["arrival"])
    for i in range(n):
        K, P, L = fake.dicts[int(sch["dict"][i])]
        Z = out["Z"][i]
        assert Z.shape == (K, int(sch["T"][i]) - L + 1)
        assert np.all(Z == float(i + 1))                     # request i's own result
    lat = out["latency_ms"]
    assert np.all(lat >= 0) and out["p50_ms"] <= out["p99_ms"] <= out["max_ms"]
    assert out["converged"] == n
    assert out["steps"] == out["gpu_launches"] == fake.launches
    assert (out["pool_peak_bytes"], out["pool_bytes"]) == (123, 456)
    assert out["throughput_req_s"] == pytest.approx(n / out["wall_s"])
    assert fake.widths == [0] * len(fake.dicts)              # the server's own widths


def test_stream_driver_passes_each_dictionary_its_segment_width():
    src = sources(1200)
    widths = [0, 63, 0, 7][:len(src)]
    fake = FakeServer(rounds=1)
    serve.run_stream(fake, FakeTorch, 4, seed=1, rate=2000.0, sources=src, T_max=600,
                     segment_widths=widths)
    assert fake.widths == widths
