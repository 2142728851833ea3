"""Command line: solve one synthetic workload on the GPU through the C ABI.

    python -m paper_1705_10087_gb300.cli --workload long_P7_K25_L64_T200000 \
        --segments 1024 --updates-per-visit 24 [--seed 0] [--tol 1e-6] [--repeat 1] \
        [--init-mode 0]
    python -m paper_1705_10087_gb300.cli --workload image_P1_K8_h8_w8_512x512

Prints one JSON line per solve with the solver statistics.  Inputs come from
paper_1705_10087_gb300.synth; lambda = 0.1 * lambda_max, for signals as
computed by the library (csc_lambda_max), for images from the cross-correlation
D~ * X taken by torch on the GPU (input preparation, outside the solver).
"""
from __future__ import annotations

import argparse
import json


def main(argv=None) -> None:
    from . import synth
    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", default="long_P7_K25_L64_T200000",
                    choices=sorted(synth.WORKLOADS) + sorted(synth.IMAGE_WORKLOADS))
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--T", type=int, default=None, help="override the signal length")
    ap.add_argument("--segments", type=int, default=0)
    ap.add_argument("--updates-per-visit", type=int, default=0)
    ap.add_argument("--tol", type=float, default=None)
    ap.add_argument("--repeat", type=int, default=1)
    ap.add_argument("--init-mode", type=int, default=0)
    a = ap.parse_args(argv)

    import torch

    from . import build, capi
    build.build()
    capi.load()
    if a.workload in synth.IMAGE_WORKLOADS:
        return image(a, synth, capi, torch)
    pb = synth.make_workload(a.workload, seed=a.seed, T=a.T)
    tol = a.tol if a.tol is not None else synth.WORKLOADS[a.workload]["tol"]
    D = torch.from_numpy(pb.D).cuda()
    X = torch.from_numpy(pb.X).cuda()
    Z = torch.zeros((pb.K, pb.Tz), dtype=torch.float32, device="cuda")
    h = capi.csc_setup(D, capi.make_opts(segments=a.segments, init_mode=a.init_mode,
                                         updates_per_visit=a.updates_per_visit))
    try:
        capi.csc_init(h, X, 1.0)
        lam = 0.1 * capi.csc_lambda_max(h)
        for _ in range(a.repeat):
            capi.csc_setup(D, capi.make_opts(segments=a.segments, init_mode=a.init_mode,
                                             updates_per_visit=a.updates_per_visit), handle=h)
            capi.csc_init(h, X, lam)
            status, E, st = capi.csc_solve(h, tol, 1 << 40, Z)
            print(json.dumps({"workload": a.workload, "seed": a.seed, "lambda": lam,
                              "status": status, "objective": E, **st}))
    finally:
        capi.csc_destroy(h)


def image(a, synth, capi, torch) -> None:
    """csc2d_solve on a synthetic image workload, automatic tiles."""
    w = synth.IMAGE_WORKLOADS[a.workload]
    pb = synth.make_image_workload(a.workload, seed=a.seed)
    tol = a.tol if a.tol is not None else w["tol"]
    D = torch.from_numpy(pb.D).cuda()
    X = torch.from_numpy(pb.X).cuda()
    # lambda_max = max |D~ * X| (Sec. 4); conv2d is the cross-correlation
    lam = 0.1 * float(torch.nn.functional.conv2d(X[None].double(), D.double()).abs().max())
    Z = torch.zeros((w["K"], w["H"] - w["h"] + 1, w["W"] - w["w"] + 1), dtype=torch.float32,
                    device="cuda")
    for _ in range(a.repeat):
        status, E, st = capi.csc2d_solve(D, X, lam, tol, updates_per_visit=a.updates_per_visit,
                                         Z_out=Z)
        print(json.dumps({"workload": a.workload, "seed": a.seed, "lambda": lam,
                          "status": status, "objective": E, **st}))


if __name__ == "__main__":
    main()
