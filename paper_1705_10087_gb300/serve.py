"""Driver of the serving engine (include/csc_server.h) for a request stream.

    python -m paper_1705_10087_gb300.serve [--requests 2000] [--rate 200] [--seed 0]

Replays the first N requests of a synthetic stream in real time: each request
is submitted when its arrival time comes, csc_server_step runs scheduling
rounds while anything is queued or active, and finished requests are fetched
(Z copied to a pinned host buffer).  Latency = completion seen by the driver
minus scheduled arrival.  Prints one JSON line with p50/p99 latency and
throughput.  All solver work runs in libcsc.so; this module only paces
arrivals and moves data.
"""
from __future__ import annotations

import argparse
import json
import time

import numpy as np

from . import synth

WORKLOAD = "serve_4dict_poisson200_T5000_2000000"


def run_stream(capi, torch, n_requests: int, seed: int = 0, rate: float | None = None,
               name: str = WORKLOAD, sources=None, T_max: int | None = None,
               budget_bytes: int | None = None, sweeps_per_step: int = 0,
               keep_Z: bool = False, workers: int = 0, segment_widths=None) -> dict:
    w = synth.SERVE_WORKLOADS[name]
    sch = synth.serve_schedule(name, n_requests, seed=seed, T_max=T_max)
    if rate is not None:
        sch["arrival"] = sch["arrival"] * (w["rate"] / rate)
    if sources is None:
        sources = synth.serve_sources(name, seed=seed, T_source=int(sch["T"].max()),
                                      workers=workers)
    budget = int(budget_bytes if budget_bytes is not None else w["budget_bytes"])
    srv = capi.csc_server_create(hbm_budget_bytes=budget, sweeps_per_step=sweeps_per_step)
    out = {"requests": n_requests, "seed": seed, "budget_bytes": budget}
    try:
        widths = list(segment_widths) if segment_widths is not None else [0] * len(sources)
        dicts = [capi.csc_server_add_dictionary(srv, pb.D, segment_width=int(wd))
                 for pb, wd in zip(sources, widths)]
        zmax = max(pb.K * (int(sch["T"].max()) - pb.L + 1) for pb in sources)
        zbuf = torch.empty(zmax, dtype=torch.float32).pin_memory()
        # request windows, cut before the clock starts
        Xs = []
        for i in range(n_requests):
            pb = sources[int(sch["dict"][i])]
            T = int(sch["T"][i])
            off = int(sch["offset_frac"][i] * (pb.T - T + 1))
            Xs.append(np.ascontiguousarray(pb.X[:, off:off + T]))
        ids = {}
        lat = np.zeros(n_requests)
        infos = [None] * n_requests
        Zs = [None] * n_requests
        nxt = 0
        steps = 0
        launches0 = capi.csc_server_kernel_launches(srv)
        t0 = time.perf_counter()
        while nxt < n_requests or ids:
            now = time.perf_counter() - t0
            while nxt < n_requests and sch["arrival"][nxt] <= now:
                rid = capi.csc_server_submit(srv, dicts[int(sch["dict"][nxt])], Xs[nxt],
                                             -w["lambda_frac"], w["tol"])
                ids[rid] = nxt
                nxt += 1
            if not ids:
                time.sleep(max(0.0, sch["arrival"][nxt] - (time.perf_counter() - t0)))
                continue
            _, _, ndone = capi.csc_server_step(srv)
            steps += 1
            if ndone:
                t_seen = time.perf_counter() - t0
                for rid in capi.csc_server_completed(srv):
                    i = ids.pop(rid)
                    pb = sources[int(sch["dict"][i])]
                    nzc = pb.K * (int(sch["T"][i]) - pb.L + 1)
                    Zv = zbuf[:nzc].view(pb.K, -1)
                    infos[i] = capi.csc_server_fetch(srv, rid, Zv)
                    if keep_Z:
                        Zs[i] = Zv.numpy().copy()
                    lat[i] = t_seen - sch["arrival"][i]
        wall = time.perf_counter() - t0
        launches = capi.csc_server_kernel_launches(srv) - launches0
        mem = capi.csc_server_memory(srv)
    finally:
        capi.csc_server_destroy(srv)
    samples = int(sch["T"].sum())
    out.update({
        "wall_s": wall, "steps": steps, "gpu_launches": launches,
        "offered_rate_req_s": n_requests / float(sch["arrival"][-1]),
        "throughput_req_s": n_requests / wall, "throughput_samples_s": samples / wall,
        "offered_samples_s": samples / float(sch["arrival"][-1]),
        "p50_ms": 1e3 * float(np.percentile(lat, 50)), "p99_ms": 1e3 * float(np.percentile(lat, 99)),
        "mean_ms": 1e3 * float(lat.mean()), "max_ms": 1e3 * float(lat.max()),
        "converged": int(sum(1 for x in infos if x and x["converged"])),
        "pool_peak_bytes": mem["peak"], "pool_bytes": mem["pool_bytes"],
    })
    out["latency_ms"] = lat * 1e3
    out["infos"] = infos
    out["Z"] = Zs
    out["schedule"] = sch
    return out


def main(argv=None) -> None:
    ap = argparse.ArgumentParser()
    ap.add_argument("--requests", type=int, default=2000)
    ap.add_argument("--rate", type=float, default=None)
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--sweeps-per-step", type=int, default=0)
    a = ap.parse_args(argv)
    import torch

    from . import build, capi
    build.build()
    capi.load()
    r = run_stream(capi, torch, a.requests, seed=a.seed, rate=a.rate,
                   sweeps_per_step=a.sweeps_per_step, workers=4)
    print(json.dumps({k: v for k, v in r.items()
                      if k not in ("latency_ms", "infos", "Z", "schedule")}))


if __name__ == "__main__":
    main()
