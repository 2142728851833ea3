#!/usr/bin/env python3
"""Benchmark: segmented locally greedy convolutional coordinate descent on GB300.

Workload (the long-signal setting of Sec. 4, at the sizes this project
targets): one multichannel signal, P = 7 channels, K = 25 unit-norm Gaussian
atoms of length L = 64, T = 200,000 samples, Bernoulli(0.005)-Gaussian
activations, noise sigma = 0.1, lambda = 0.1 lambda_max, stopping rule
max |Delta Z| < 1e-6 followed by the FP64 beta re-synchronisation.  Inputs
are synthetic and seeded (rank r solves seed r: weak scaling, no collective
on the data path).

One step = csc_setup (DtD, norms) + csc_init (beta = D~*X) + csc_solve (phase
schedule to convergence, FP64 resync, FP64 objective), inputs resident in
HBM.  The problem state (about 60 MB) fits in L2, so L2 is flushed (a 256 MB
write) between timed steps, outside the timed intervals.

Printed: one JSON line.  value = applied coordinate updates per second of
whole step time (summed over ranks / max over ranks of the time).
time_to_gap_ms is the time from the step start until the objective is within
a relative 1e-4 of the optimum E* stored in tests/golden/optimum.json (written
by the FP64 oracle).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "time to 1e-4 objective gap & CD updates/s vs plain GPU; serve p50/p99 ms"
WORKLOAD = "long_P7_K25_L64_T200000"
GOLDEN = os.path.join(ROOT, "tests", "golden", "optimum.json")
HBM_FALLBACK_GBS = 6800.0


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--segments", type=int, default=1024)
    ap.add_argument("--updates-per-visit", type=int, default=24)
    ap.add_argument("--no-sweep", action="store_true", help="skip the segment-count sweep")
    ap.add_argument("--tol", type=float, default=1e-6)
    ap.add_argument("--threads-per-segment", type=int, default=0, choices=[0, 32, 128],
                    help="phase kernel form: 0 automatic, 32 one warp per segment, 128 a block")
    ap.add_argument("--init-mode", type=int, default=0,
                    help="beta0 kernel: 0 automatic (tensor cores where their tile needs at "
                         "most half the shared memory, else FP32), 1 tensor cores (split BF16), "
                         "2 one BF16 product, 3 FP32 compensated")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-batch", action="store_true",
                    help="skip the 512-signal batched-vs-plain comparison")
    ap.add_argument("--no-serve", action="store_true", help="skip the request-stream leg")
    ap.add_argument("--no-verylong", action="store_true",
                    help="skip the very long recording (T = 5e6) leg")
    ap.add_argument("--no-image", action="store_true", help="skip the 2-D image leg")
    ap.add_argument("--serve-requests", type=int, default=400)
    return ap.parse_args()


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return HBM_FALLBACK_GBS, "fallback"


def golden(seed: int):
    try:
        with open(GOLDEN) as f:
            return json.load(f).get(f"{WORKLOAD}/seed{seed}")
    except OSError:
        return None


def input_hash(pb) -> str:
    import hashlib
    h = hashlib.sha256()
    h.update(pb.D.tobytes())
    h.update(pb.X.tobytes())
    return h.hexdigest()[:16]


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled every 200 ms."""

    FIELDS = ("timestamp,index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []
        self.window = None  # (start, end) wall-clock seconds of the timed region

    def mark(self, start: float, end: float):
        self.window = (start, end)

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-i", str(self.gpu), "-lms", "50"], stdout=subprocess.PIPE,
                stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.thread.join(timeout=2)

    def summary(self):
        import datetime
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 10:
                continue
            try:
                ts = datetime.datetime.strptime(f[0], "%Y/%m/%d %H:%M:%S.%f").timestamp()
                clk, cmax = float(f[2]), float(f[3])
            except ValueError:
                continue
            # samples inside the timed region only (50 ms sampling period)
            if self.window and not (self.window[0] - 0.05 <= ts <= self.window[1] + 0.05):
                continue
            sm.append(clk)
            mx = cmax
            for n, v in zip(names, f[6:10]):
                if v.lower() == "active":
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": mx, "reasons": ["unavailable"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def phase_profile():
    """Per-launch counters of the phase kernel from the committed ncu summary
    (dram_bytes_per_launch, l2_bytes_per_launch, l2_throughput_pct), or {}
    when the kernel source changed since those counters were taken."""
    import hashlib
    try:
        text = open(os.path.join(ROOT, "profiles", f"phase_kernel_{WORKLOAD}.md")).read()
        src = open(os.path.join(ROOT, "paper_1705_10087_gb300", "csrc", "kernel_phase.cu"), "rb").read()
    except OSError:
        return {}
    fields = dict(ln.split(":", 1) for ln in text.splitlines()
                  if ln.startswith(("kernel_source", "dram_", "l2_")))
    if fields.get("kernel_source_sha256_16", "").strip() != hashlib.sha256(src).hexdigest()[:16]:
        return {}
    out = {}
    for k in ("dram_bytes_per_launch", "l2_bytes_per_launch", "l2_throughput_pct"):
        try:
            out[k] = float(fields[k])
        except (KeyError, ValueError):
            pass
    return out


def over_ranks(dist, device, elapsed, units):
    """Whole-job figures of N independent replicas: the slowest rank's elapsed
    time (max over ranks) and the units all ranks processed (sum); without a
    process group, this rank's own."""
    if dist is None:
        return float(elapsed), float(units)
    import torch
    t = torch.tensor([float(elapsed)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    u = torch.tensor([float(units)], dtype=torch.float64, device=device)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return float(t.item()), float(u.item())


def time_to_gap_ms(trace, init_ms, E_star, rel=1e-4):
    E = trace["E_start"] - np.cumsum(trace["decrease"])
    ok = np.nonzero((E - E_star) <= rel * E_star)[0]
    if ok.size == 0:
        return None
    # first launch reaching the gap; launches without updates carry no time stamp
    t = trace["t_ns"][: ok[0] + 1]
    t = t[t >= 0]
    return init_ms + (float(t[-1]) / 1e6 if t.size else 0.0)


BATCH = "batch_P7_K25_L64_n512_T10000_500000"
GOLDEN_BATCH = os.path.join(ROOT, "tests", "golden", "optimum_batch.json")


def batch_leg(args, capi, torch):
    """The 512-signal batch solved two ways to the same accuracy: batched (all
    signals in one csc_init_batch + csc_solve) and plain (one csc_init +
    csc_solve per signal, one handle, signals one after another).

    For each way, the time to a relative objective gap <= 1e-4 on EVERY signal
    is the solve time at the largest stopping tolerance (from a fixed grid)
    whose solution meets that gap against E*_i of tests/golden/optimum_batch.json
    (FP64 oracle); time = csc_init + csc_solve of all signals (CUDA events)."""
    import hashlib
    from paper_1705_10087_gb300 import batch, synth
    t0 = time.perf_counter()
    pbs = synth.make_batch(BATCH, seed=0, workers=min(16, os.cpu_count() or 1))
    gen_s = time.perf_counter() - t0
    D = pbs[0].D
    X, T = batch.pack([pb.X for pb in pbs])
    K, L = D.shape[0], D.shape[2]
    n = len(pbs)
    try:
        with open(GOLDEN_BATCH) as f:
            gb = json.load(f)
        h = hashlib.sha256()
        h.update(D.tobytes())
        for pb in pbs:
            h.update(hashlib.sha256(pb.X.tobytes()).hexdigest().encode())
        if h.hexdigest()[:16] != gb["input_sha256_16"]:
            gb = None
    except (OSError, KeyError, ValueError):
        gb = None
    if gb is None:
        return {"workload": BATCH, "unavailable": "no stored optimum for these inputs"}
    lam = np.array(gb["lambda"])
    E_star = np.array(gb["E_star"])
    Dd = torch.from_numpy(D).cuda()
    Xd = torch.from_numpy(X).cuda()
    Xi = [torch.from_numpy(np.ascontiguousarray(pb.X)).cuda() for pb in pbs]
    del pbs
    Tz = int(T.sum()) - L + 1
    Zd = torch.zeros((K, Tz), dtype=torch.float32, device="cuda")
    Zi = torch.zeros(K * (int(T.max()) - L + 1), dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()
    # autotune (segment width, updates per visit) on the first 32 signals
    a = batch.offsets(T)
    nt = min(32, n)
    ht = capi.csc_setup(Dd, capi.make_opts(updates_per_visit=args.updates_per_visit))
    try:
        capi.csc_init_batch(ht, Xd[:, :int(a[nt])].contiguous(), T[:nt], lam[:nt])
        tune = capi.csc_autotune(ht, args.tol)
    finally:
        capi.csc_destroy(ht)
    u, wseg, tps = tune["updates_per_visit"], tune["segment_width"], tune["threads_per_segment"]

    def batched(tol):
        hb = capi.csc_setup(Dd, capi.make_opts(updates_per_visit=u, segment_width=wseg,
                                               threads_per_segment=tps))
        try:
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            capi.csc_init_batch(hb, Xd, T, lam)
            status, E, st = capi.csc_solve(hb, tol, 1 << 40, Zd)
            e1.record(stream)
            torch.cuda.synchronize()
            Es = capi.csc_get_objectives(hb, n)
            return e0.elapsed_time(e1), Es, st["updates"], status
        finally:
            capi.csc_destroy(hb)

    def plain(tol):
        hp = capi.csc_setup(Dd, capi.make_opts(updates_per_visit=u, segment_width=wseg,
                                               threads_per_segment=tps))
        try:
            Es = np.zeros(n)
            ups = 0
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            worst = capi.CSC_OK
            for i in range(n):
                capi.csc_init(hp, Xi[i], float(lam[i]))
                status, E, st = capi.csc_solve(hp, tol, 1 << 40,
                                               Zi[:K * (int(T[i]) - L + 1)].view(K, -1))
                Es[i] = E
                ups += st["updates"]
                worst = max(worst, status)
            e1.record(stream)
            torch.cuda.synchronize()
            return e0.elapsed_time(e1), Es, ups, worst
        finally:
            capi.csc_destroy(hp)

    out = {"workload": BATCH, "signals": n, "samples": int(T.sum()), "P": 7, "K": K, "L": L,
           "updates_per_visit": u, "segment_width": wseg, "threads_per_segment": tps,
           "autotune": tune, "gen_s": gen_s,
           "gap_target": 1e-4, "E_star": "FP64 oracle per signal (stored)"}
    grid = (1e-1, 3e-2, 1e-2, 3e-3, 1e-3, 3e-4, 1e-4, 1e-5, 1e-6)
    for name, fn in (("batched", batched), ("plain", plain)):
        fn(grid[0])  # warm-up (module load, allocations)
        res = None
        for tol in grid:
            ms, Es, ups, status = min((fn(tol) for _ in range(2)), key=lambda r: r[0])
            gap = float(np.max((Es - E_star) / E_star))
            if gap <= 1e-4:
                res = {"tol": tol, "ms": ms, "max_rel_gap": gap, "updates": ups,
                       "updates_per_s": ups / (ms * 1e-3), "status": status}
                break
        ms6, Es6, ups6, st6 = min((fn(1e-6) for _ in range(2)), key=lambda r: r[0]) \
            if res is None or res["tol"] != 1e-6 else (res["ms"], None, res["updates"],
                                                         res["status"])
        out[name] = {"time_to_gap": res, "converged_tol_1e-6_ms": ms6,
                     "converged_updates": ups6}
    if out["batched"]["time_to_gap"] and out["plain"]["time_to_gap"]:
        out["speedup_time_to_gap"] = (out["plain"]["time_to_gap"]["ms"] /
                                      out["batched"]["time_to_gap"]["ms"])
    out["speedup_converged"] = (out["plain"]["converged_tol_1e-6_ms"] /
                                out["batched"]["converged_tol_1e-6_ms"])
    return out


def serve_leg(args, capi, torch):
    """The request stream (Poisson arrivals at 200 req/s, lengths log-uniform in
    [5e3, 2e6], four resident dictionaries, 40 GB pool, tol 1e-3, which meets
    the 1e-4 objective-gap target on the oracle-checked samples) replayed in
    real time through the serving engine: the first N requests at the offered
    rate, and the same requests at a tenth of it."""
    from paper_1705_10087_gb300 import serve, synth
    name = serve.WORKLOAD
    w = synth.SERVE_WORKLOADS[name]
    n = args.serve_requests
    sch = synth.serve_schedule(name, n, seed=0)
    sources = synth.serve_sources(name, seed=0, T_source=int(sch["T"].max()),
                                  workers=min(4, os.cpu_count() or 1))
    out = {"workload": name, "requests": n, "tol": w["tol"], "lambda": "0.1*lambda_max",
           "budget_bytes": w["budget_bytes"], "dictionaries_KLP": [list(d) for d in w["dicts"]]}
    for label, rate in (("offered", w["rate"]), ("tenth", w["rate"] / 10)):
        r = serve.run_stream(capi, torch, n, seed=0, rate=rate, sources=sources)
        out[label] = {k: r[k] for k in ("offered_rate_req_s", "offered_samples_s", "wall_s",
                                         "throughput_req_s", "throughput_samples_s", "p50_ms",
                                         "p99_ms", "mean_ms", "max_ms", "converged", "steps",
                                         "gpu_launches", "pool_peak_bytes")}
        # per dictionary p50 / p99
        lat = r["latency_ms"]
        out[label]["per_dictionary"] = {
            str(j): {"n": int((sch["dict"] == j).sum()),
                     "p50_ms": float(np.percentile(lat[sch["dict"] == j], 50)),
                     "p99_ms": float(np.percentile(lat[sch["dict"] == j], 99))}
            for j in range(len(w["dicts"])) if (sch["dict"] == j).any()}
    return out


VERYLONG = "verylong_P1_K25_L200_T5000000"


def verylong_leg(args, capi, torch):
    """The very long recording (P=1, K=25, L=200, T=5e6, about 1.4 h at 1 kHz)
    with the default options (tensor-core beta0, segments of 2L-2 columns,
    u = 24), tol 1e-6, and again with the options csc_autotune picks for it
    ("autotuned").  Per run: csc_setup + csc_init + csc_solve timed with
    CUDA events; the beta0 kernel alone by the library's own event pair
    (csc_init_time); time to a 1e-4 relative gap against the oracle's E*
    stored by tests/golden/make_golden.py --verylong.  The state (beta0, r,
    Z: 1.5 GB) is far larger than L2."""
    from paper_1705_10087_gb300 import synth
    pb = synth.make_workload(VERYLONG, seed=0)
    try:
        with open(GOLDEN) as f:
            g = json.load(f).get(f"{VERYLONG}/seed0")
    except OSError:
        g = None
    if g is not None and g.get("input_sha256_16") != input_hash(pb):
        g = None
    stream = torch.cuda.current_stream()
    D = torch.from_numpy(pb.D).cuda()
    X = torch.from_numpy(pb.X).cuda()
    Z = torch.zeros((pb.K, pb.Tz), dtype=torch.float32, device="cuda")
    opts = capi.make_opts(updates_per_visit=24, time_kernels=1)
    h = capi.csc_setup(D, opts)
    if g is not None:
        lam = g["lambda"]
    else:
        capi.csc_init(h, X, 1.0)
        lam = 0.1 * capi.csc_lambda_max(h)
    def timed_runs(opts):
        runs = []
        for i in range(4):  # the first run warms up
            ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
            ev[0].record(stream)
            capi.csc_setup(D, opts, handle=h)
            capi.csc_init(h, X, lam)
            ev[1].record(stream)
            status, E, st = capi.csc_solve(h, args.tol, 1 << 40, Z)
            ev[2].record(stream)
            torch.cuda.synchronize()
            b0 = capi.csc_init_time(h)
            tr = capi.csc_get_trace(h)
            init_ms = ev[0].elapsed_time(ev[1])
            if i > 0:
                runs.append({"step_ms": ev[0].elapsed_time(ev[2]), "init_ms": init_ms,
                             "beta0_kernel_ms": b0, "solve_ms": st["solve_ms"],
                             "updates": st["updates"], "status": status,
                             "resyncs": st["resyncs"], "segments": st["segments"],
                             "time_to_gap_ms": time_to_gap_ms(tr, init_ms, g["E_star"]) if g else None,
                             "rel_gap_final": (E - g["E_star"]) / g["E_star"] if g else None})
        return min(runs, key=lambda r: r["step_ms"]), len(runs)

    best, nruns = timed_runs(opts)
    # the same recording with the library's autotuner choosing the segment
    # width, u and threads per segment for this (K, L, P) (tuned outside the
    # timed runs)
    capi.csc_init(h, X, lam)
    tune = capi.csc_autotune(h, args.tol)
    topts = capi.make_opts(segment_width=tune["segment_width"],
                           updates_per_visit=tune["updates_per_visit"],
                           threads_per_segment=tune["threads_per_segment"], time_kernels=1)
    tuned, _ = timed_runs(topts)
    tuned.update({"segment_width": tune["segment_width"],
                  "updates_per_visit": tune["updates_per_visit"],
                  "threads_per_segment": tune["threads_per_segment"],
                  "updates_per_s": tuned["updates"] / (tuned["step_ms"] * 1e-3)})
    capi.csc_destroy(h)
    peak, kind = peaks()
    # beta0 kernel: X read once; beta0, the cold-start r and the cold-start
    # Z = 0 written
    b0_bytes = 4.0 * pb.P * pb.T + 3 * 4.0 * pb.K * pb.Tz
    b0_gbs = b0_bytes / (best["beta0_kernel_ms"] * 1e-3) / 1e9 if best["beta0_kernel_ms"] > 0 else None
    return {"workload": VERYLONG, "P": pb.P, "K": pb.K, "L": pb.L, "T": pb.T, "tol": args.tol,
            "lambda": "0.1*lambda_max", "runs": nruns, **best, "autotuned": tuned,
            "updates_per_s": best["updates"] / (best["step_ms"] * 1e-3),
            "solve_updates_per_s": best["updates"] / (best["solve_ms"] * 1e-3),
            "beta0_roofline": {"bound": "hbm", "bytes": b0_bytes, "achieved_gbs": b0_gbs,
                               "peak_gbs": peak, "peak_kind": kind,
                               "frac": b0_gbs / peak if b0_gbs else None}}


IMAGE = "image_P1_K8_h8_w8_512x512"


def image_leg(args, capi, torch):
    """The 2-D variant: one 512 x 512 gray image, K = 8 atoms of 8 x 8, the Sec. 4
    law; csc2d_solve to tol 1e-6 with automatic tiles (row bands of 2h-2 rows cut
    into column blocks of 2w-2 columns), timed with CUDA events around the call
    (setup, beta0, tile phases, resyncs, objective), against the 2-D oracle's E*
    stored by tests/golden/make_golden.py --image2d."""
    from paper_1705_10087_gb300 import synth
    pb = synth.make_image_workload(IMAGE, seed=0)
    try:
        with open(GOLDEN) as f:
            g = json.load(f).get(f"{IMAGE}/seed0")
    except OSError:
        g = None
    if g is None or g.get("input_sha256_16") != input_hash(pb):
        return {"workload": IMAGE, "unavailable": "no stored optimum for these inputs"}
    w = synth.IMAGE_WORKLOADS[IMAGE]
    stream = torch.cuda.current_stream()
    D = torch.from_numpy(pb.D).cuda()
    X = torch.from_numpy(pb.X).cuda()
    Hz, Wz = w["H"] - w["h"] + 1, w["W"] - w["w"] + 1
    Z = torch.zeros((w["K"], Hz, Wz), dtype=torch.float32, device="cuda")
    runs = []
    for i in range(4):  # the first run warms up
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        status, E, st = capi.csc2d_solve(D, X, g["lambda"], w["tol"], Z_out=Z)
        e1.record(stream)
        torch.cuda.synchronize()
        if i > 0:
            runs.append({"ms": e0.elapsed_time(e1), "solve_ms": st["solve_ms"], "status": status,
                         "updates": st["updates"], "sweeps": st["sweeps"], "bands": st["bands"],
                         "col_blocks": st["col_blocks"], "phases": st["phases"],
                         "resyncs": st["resyncs"],
                         "rel_gap_final": (E - g["E_star"]) / g["E_star"]})
    best = min(runs, key=lambda r: r["ms"])
    return {"workload": IMAGE, "K": w["K"], "P": w["P"], "h": w["h"], "w": w["w"],
            "H": w["H"], "W": w["W"], "tol": w["tol"], "lambda": "0.1*lambda_max",
            **best, "updates_per_s": best["updates"] / (best["ms"] * 1e-3)}


def cpu_baseline(pb, lam, tol, M, u):
    """The FP64 oracle as it stands (single thread), on the full problem."""
    import oracle
    t = time.perf_counter()
    r = oracle.locally_greedy_cd(pb.D, pb.X, lam, tol, M=M, mode="phase", updates_per_visit=u)
    dt = time.perf_counter() - t
    return {"value": r["n_updates"] / dt, "unit": "updates/s", "cores": 1, "kind": "oracle",
            "sample": f"full solve (DtD, D~*X, phase-schedule CD to max|dZ|<{tol:g}) of seed 0, "
                      f"M={M}, u={u}: {r['n_updates']} updates in {dt:.2f} s"}


def cpu_baseline_multicore(pb, lam, tol, M, u):
    """The same phase-schedule solve with the segments of a phase spread over
    all host cores (oracle/csc_baseline_omp.c: identical results to the
    oracle, the CPU analogue of DICOD)."""
    from oracle import baseline_omp
    cores = os.cpu_count() or 1
    t = time.perf_counter()
    r = baseline_omp.phase_cd(pb.D, pb.X, lam, tol, M, u, threads=cores)
    dt = time.perf_counter() - t
    return {"value": r["n_updates"] / dt, "unit": "updates/s", "cores": r["threads"],
            "kind": "oracle phase schedule, OpenMP over the segments of a phase",
            "solve_s": dt,
            "sample": f"full solve (DtD, D~*X, phase-schedule CD to max|dZ|<{tol:g}) of seed 0, "
                      f"M={M}, u={u}: {r['n_updates']} updates in {dt:.2f} s on "
                      f"{r['threads']} threads"}


def run_reference(args):
    """CPU oracle arm: rank 0 only; each step is the oracle's solve of seed 0,
    bounded to 30,000 updates so that warmup + steps stay within minutes."""
    if int(os.environ.get("RANK", "0")) != 0:
        return
    from paper_1705_10087_gb300 import synth
    import oracle
    pb = synth.make_workload(WORKLOAD, seed=0)
    g = golden(0)
    lam = g["lambda"] if g else 0.1 * oracle.lambda_max(pb.D, pb.X)
    cap = 30_000
    times, ups = [], []
    for i in range(args.warmup + args.steps):
        t = time.perf_counter()
        r = oracle.locally_greedy_cd(pb.D, pb.X, lam, args.tol, M=args.segments, mode="phase",
                                     updates_per_visit=args.updates_per_visit, max_updates=cap)
        dt = time.perf_counter() - t
        if i >= args.warmup:
            times.append(dt)
            ups.append(r["n_updates"])
    v = sum(ups) / sum(times)
    sample = (f"per step: oracle setup + D~*X + first {cap} updates of the phase-schedule "
              f"solve (M={args.segments}) of seed 0, 1 thread")
    print(json.dumps({
        "metric": METRIC, "value": v, "unit": "updates/s", "impl": "reference",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * sum(times) / len(times), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "P": 7, "K": 25, "L": 64, "T": 200_000,
                   "segments": args.segments, "updates_per_visit": args.updates_per_visit,
                   "tol": args.tol},
        "cpu_baseline": {"value": v, "unit": "updates/s", "cores": 1, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": v, "unit": "updates/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0}}))


def sharded_main(args, torch, dist, world, rank):
    """N > 1: one signal of N x 200,000 samples (the long workload's recipe,
    seed 0) cut into N shards, one per rank, solved by DICOD's protocol
    (paper_1705_10087_gb300/shard.py): per phase each rank runs its segments
    and exchanges its [K][L-1] halo with its neighbours over NCCL (device
    buffers); a sweep without update on any rank ends a round; exact resyncs
    and the objective are reduced over ranks.  Per-rank work is fixed as N
    grows (weak scaling); value = updates of all ranks / slowest rank's time."""
    from paper_1705_10087_gb300 import build, capi, shard, synth
    build.build()
    capi.load()
    T1 = synth.WORKLOADS[WORKLOAD]["T"]
    pb = synth.make_workload(WORKLOAD, seed=0, T=world * T1)
    M = args.segments * world
    plan = capi.csc_shard_plan_make(pb.T, pb.L, M, world, rank)
    a0, n0 = plan["x_first"], plan["x_count"]
    Xw = torch.from_numpy(np.ascontiguousarray(pb.X[:, a0:a0 + n0])).cuda()
    D = torch.from_numpy(pb.D).cuda()
    opts = capi.make_opts(updates_per_visit=args.updates_per_visit, init_mode=args.init_mode)
    h = capi.csc_setup(D, opts)
    comm = shard.TorchComm(dist, device="cuda")
    capi.csc_shard_init(h, plan, Xw, 1.0)
    lam = 0.1 * comm.max(capi.csc_lambda_max(h))  # lambda_max over the whole signal
    make = lambda shape: torch.zeros(shape, dtype=torch.float32, device="cuda")  # noqa: E731
    stream = torch.cuda.current_stream()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")

    def step():
        capi.csc_setup(D, opts, handle=h)
        capi.csc_shard_init(h, plan, Xw, lam)
        return shard.solve(shard.CapiShard(capi, h, plan), comm, pb.K, plan, args.tol, make=make)

    for _ in range(args.warmup):
        step()
        flush.zero_()
    torch.cuda.synchronize()
    dist.barrier()
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    tot_ms, ups = 0.0, 0
    res = None
    for _ in range(args.steps):
        flush.zero_()
        ev0.record(stream)
        res = step()
        ev1.record(stream)
        torch.cuda.synchronize()
        tot_ms += ev0.elapsed_time(ev1)
        ups += capi.csc_shard_updates(h)  # this rank's updates of the step
    dist.barrier()
    torch.cuda.synchronize()
    t_max, u_all = over_ranks(dist, "cuda", tot_ms, ups)
    # end to end: host (pinned) samples in, host Z out, through the same calls
    Xh = torch.from_numpy(np.ascontiguousarray(pb.X[:, a0:a0 + n0])).pin_memory()
    Zh = torch.zeros((pb.K, plan["col_count"]), dtype=torch.float32).pin_memory()
    e_t, e_u = 0.0, 0
    for _ in range(args.steps):
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        capi.csc_setup(D, opts, handle=h)
        capi.csc_shard_init(h, plan, Xh, lam)
        shard.solve(shard.CapiShard(capi, h, plan), comm, pb.K, plan, args.tol, make=make)
        capi.csc_shard_get_z(h, Zh)
        e_t += time.perf_counter() - t0
        e_u += capi.csc_shard_updates(h)
    e_tmax, e_uall = over_ranks(dist, "cuda", e_t, e_u)
    capi.csc_destroy(h)
    if rank == 0:
        print(json.dumps({
            "metric": METRIC, "value": u_all / (t_max * 1e-3), "unit": "updates/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": t_max / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": f"{WORKLOAD} per rank: one signal of {world} x {T1} samples "
                                   f"in {world} shards", "P": pb.P, "K": pb.K, "L": pb.L,
                       "T": pb.T, "segments": M, "updates_per_visit": args.updates_per_visit,
                       "tol": args.tol, "lambda": "0.1*lambda_max",
                       "l2": "flushed between steps (256 MB write)",
                       "parallelism": f"shards x{world}: halo exchange per phase over NCCL"},
            "converged": bool(res["converged"]), "sweeps": res["sweeps"],
            "resyncs": res["resyncs"], "objective": res["E"],
            "e2e": {"value": e_uall / e_tmax, "unit": "updates/s",
                    "h2d_bytes_per_step": int(4 * pb.P * n0),
                    "d2h_bytes_per_step": int(4 * pb.K * plan["col_count"])}}))
    dist.destroy_process_group()


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)

    import torch
    import torch.distributed as dist

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA device (the solver has no CPU path)")
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
        return sharded_main(args, torch, dist, world, rank)

    from paper_1705_10087_gb300 import build, capi, synth
    build.build()
    capi.load()

    pb = synth.make_workload(WORKLOAD, seed=rank)
    g = golden(rank)
    if g is not None and g.get("input_sha256_16") != input_hash(pb):
        g = None  # generator does not reproduce the stored inputs on this machine
    stream = torch.cuda.current_stream()
    D = torch.from_numpy(pb.D).cuda()
    X = torch.from_numpy(pb.X).cuda()
    Z = torch.zeros((pb.K, pb.Tz), dtype=torch.float32, device="cuda")
    opts = capi.make_opts(segments=args.segments, updates_per_visit=args.updates_per_visit,
                          time_kernels=1, init_mode=args.init_mode,
                          threads_per_segment=args.threads_per_segment)
    h = capi.csc_setup(D, opts)
    if g is not None:
        lam = g["lambda"]
    else:
        capi.csc_init(h, X, 1.0)
        lam = 0.1 * capi.csc_lambda_max(h)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")

    def step(ev):
        ev[0].record(stream)
        capi.csc_setup(D, opts, handle=h)
        capi.csc_init(h, X, lam)
        ev[1].record(stream)
        status, E, st = capi.csc_solve(h, args.tol, 1 << 40, Z)
        ev[2].record(stream)
        if status != capi.CSC_OK:
            raise RuntimeError(f"solve did not converge: {st}")
        st["beta0_ms"] = capi.csc_init_time(h)  # (after the solve: no extra wait)
        return E, st

    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(3)]
           for _ in range(args.warmup + args.steps)]
    for i in range(args.warmup):
        step(evs[i])
        flush.zero_()
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    phys = os.environ.get("CUDA_VISIBLE_DEVICES", "").split(",")
    gpu_index = int(phys[local]) if phys and phys[0] not in ("",) and phys[local].isdigit() else local
    launches0 = capi.csc_kernel_launches(h)
    sts, Es = [], []
    with ClockSampler(gpu_index) as clk:
        time.sleep(0.3)  # let the sampler start
        w0 = time.time()
        for i in range(args.warmup, args.warmup + args.steps):
            E, st = step(evs[i])
            sts.append(st)
            Es.append(E)
            flush.zero_()
        torch.cuda.synchronize()
        clk.mark(w0, time.time())
    launches = capi.csc_kernel_launches(h) - launches0
    trace = capi.csc_get_trace(h)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()

    step_ms = [evs[i][0].elapsed_time(evs[i][2]) for i in range(args.warmup, args.warmup + args.steps)]
    init_ms = [evs[i][0].elapsed_time(evs[i][1]) for i in range(args.warmup, args.warmup + args.steps)]
    tot_ms = sum(step_ms)
    updates = sum(s["updates"] for s in sts)
    phase_ms = sum(s["phase_ms"] for s in sts)
    phase_launches = sum(s["phase_launches"] for s in sts)
    visits = sum(s["visits"] for s in sts)

    # algorithmic bytes of the phase kernel: per visit the segment's beta window
    # and Z in and out (16 K (w + 2L - 2)), per update one DtD column (4 K (2L-1))
    K, L = pb.K, pb.L
    w = pb.Tz / args.segments
    alg_bytes = visits * 16.0 * K * (w + 2 * L - 2) + updates * 4.0 * K * (2 * L - 1)
    achieved = alg_bytes / (phase_ms * 1e-3) / 1e9 if phase_ms > 0 else None
    peak, peak_kind = peaks()

    tot_ms_max, updates_all = over_ranks(dist if world > 1 else None, "cuda", tot_ms, updates)

    ttg = time_to_gap_ms(trace, init_ms[-1], g["E_star"]) if g else None

    # end to end through the public API with host buffers (pinned), copies inside
    Dh = torch.from_numpy(pb.D).pin_memory()
    Xh = torch.from_numpy(pb.X).pin_memory()
    Zh = torch.zeros((pb.K, pb.Tz), dtype=torch.float32).pin_memory()
    e2e_t, e2e_u = 0.0, 0
    for i in range(args.steps):
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        capi.csc_setup(Dh, opts, handle=h)
        capi.csc_init(h, Xh, lam)
        status, E, st = capi.csc_solve(h, args.tol, 1 << 40, Zh)
        e2e_t += time.perf_counter() - t0
        e2e_u += st["updates"]
    # the workload's segment-count sweep (not part of the timed steps)
    sweep = {}
    if world == 1 and not args.no_sweep:
        for M in (64, 256, 1024, 3072):
            o = capi.make_opts(segments=M, updates_per_visit=args.updates_per_visit,
                               threads_per_segment=args.threads_per_segment)
            best = None
            for _ in range(3):
                capi.csc_setup(D, o, handle=h)
                capi.csc_init(h, X, lam)
                status, E, st = capi.csc_solve(h, args.tol, 1 << 40, Z)
                tr = capi.csc_get_trace(h)
                if best is None or st["solve_ms"] < best["solve_ms"]:
                    best = {"solve_ms": st["solve_ms"], "updates": st["updates"],
                            "updates_per_s": st["updates"] / (st["solve_ms"] * 1e-3),
                            "sweeps": st["sweeps"], "phases": st["phases"],
                            "time_to_gap_solve_ms": time_to_gap_ms(tr, 0.0, g["E_star"]) if g else None,
                            "rel_gap_final": (E - g["E_star"]) / g["E_star"] if g else None}
            sweep[str(M)] = best
    capi.csc_destroy(h)
    e2e_t_max, e2e_u_all = over_ranks(dist if world > 1 else None, "cuda", e2e_t, e2e_u)
    e2e_value = e2e_u_all / e2e_t_max

    if rank != 0:
        dist.destroy_process_group() if world > 1 else None
        return
    clk_sum = clk.summary()
    prof = phase_profile()
    sm_mhz = clk_sum.get("sm_mhz") or 0.0
    line = {
        "metric": METRIC, "value": updates_all / (tot_ms_max * 1e-3), "unit": "updates/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": tot_ms_max / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOAD, "P": 7, "K": 25, "L": 64, "T": 200_000,
                   "segments": args.segments, "updates_per_visit": args.updates_per_visit,
                   "phases": sts[-1]["phases"], "tol": args.tol, "init_mode": args.init_mode,
                   "threads_per_segment": args.threads_per_segment,
                   "lambda": "0.1*lambda_max", "l2": "flushed between steps (256 MB write)",
                   "parallelism": f"replicas x{world}, one signal per GPU"},
        "time_to_gap_ms": ttg,
        "init_ms": statistics.mean(init_ms),
        "solve_ms": statistics.mean(s["solve_ms"] for s in sts),
        "updates_per_step": updates / args.steps,
        # live device time of a step by part (CUDA events inside the library)
        "breakdown_ms": {"setup_and_init": statistics.mean(init_ms),
                         "beta0_kernel": statistics.mean(s["beta0_ms"] for s in sts),
                         "phase_kernels": phase_ms / args.steps,
                         "resyncs": sum(s["resync_ms"] for s in sts) / args.steps,
                         "objective": sum(s["objective_ms"] for s in sts) / args.steps,
                         "solve_total": statistics.mean(s["solve_ms"] for s in sts)},
        "sweeps": sts[-1]["sweeps"], "resyncs": sts[-1]["resyncs"],
        "rel_gap_final": (Es[-1] - g["E_star"]) / g["E_star"] if g else None,
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak if achieved else None,
                     "traffic": prof.get("dram_bytes_per_launch"),
                     "kernel": "phase_kernel", "peak_kind": peak_kind,
                     "avg_launch_us": 1e3 * phase_ms / phase_launches if phase_launches else None,
                     "launches": phase_launches,
                     # the state lives in L2: the level the data are served from
                     "l2": {"bytes_per_launch": prof.get("l2_bytes_per_launch"),
                            "throughput_pct_of_peak": prof.get("l2_throughput_pct"),
                            "source": "ncu summary in profiles/ (null if the kernel changed)"},
                     # latency: SM cycles of phase-kernel time per applied update
                     # (all SMs together), phase time x median SM clock / updates
                     "cycles_per_update": (phase_ms * 1e-3 * sm_mhz * 1e6 / updates
                                           if updates and sm_mhz else None)},
        "gpu_launches": launches,
        "e2e": {"value": e2e_value, "unit": "updates/s",
                "h2d_bytes_per_step": int(pb.D.nbytes + pb.X.nbytes),
                "d2h_bytes_per_step": int(pb.K * pb.Tz * 4 + 8)},
        "clocks": clk_sum,
    }
    if sweep:
        line["segment_sweep"] = sweep

    def leg(fn):
        # a secondary leg that fails is reported in its own key; the headline
        # measurement above stands
        try:
            return fn(args, capi, torch)
        except Exception as e:  # noqa: BLE001 (any failure of the leg)
            return {"error": f"{type(e).__name__}: {e}"}

    if world == 1 and not args.no_verylong:
        line["verylong"] = leg(verylong_leg)
    if world == 1 and not args.no_image:
        line["image2d"] = leg(image_leg)
    if world == 1 and not args.no_batch:
        line["batch"] = leg(batch_leg)
    if world == 1 and not args.no_serve:
        line["serve"] = leg(serve_leg)
    if world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(pb, lam, args.tol, args.segments,
                                            args.updates_per_visit)
        line["cpu_baseline_multicore"] = cpu_baseline_multicore(
            pb, lam, args.tol, args.segments, args.updates_per_visit)
    print(json.dumps(line))
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
