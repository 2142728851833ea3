"""Write the stored reference values of the benchmark workloads.

Calls only the FP64 oracle (oracle/) on inputs from the seeded generator:
for each (workload, seed) it records lambda = 0.1 * lambda_max, the optimum
E* = E(Z*) reached by the oracle's phase-schedule locally greedy CD at
eps = 1e-10, and a hash of the generated inputs so a reader can tell when
the generator no longer reproduces them.

    python tests/golden/make_golden.py            # all entries
"""
import hashlib
import json
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import oracle  # noqa: E402
from paper_1705_10087_gb300 import synth  # noqa: E402

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "optimum.json")
ENTRIES = [("long_P7_K25_L64_T200000", s, 1024) for s in range(8)] + \
          [("short_P1_K5_L16_T2000", 0, 1)]


def input_hash(pb) -> str:
    h = hashlib.sha256()
    h.update(pb.D.tobytes())
    h.update(pb.X.tobytes())
    return h.hexdigest()[:16]


def main():
    res = {}
    for name, seed, M in ENTRIES:
        t = time.time()
        pb = synth.make_workload(name, seed=seed)
        lmax = oracle.lambda_max(pb.D, pb.X)
        lam = 0.1 * lmax
        r = oracle.locally_greedy_cd(pb.D, pb.X, lam, 1e-10, M=M, mode="phase")
        assert r["converged"]
        E = oracle.objective(pb.D, pb.X, r["Z"], lam)
        res[f"{name}/seed{seed}"] = {
            "lambda": lam, "lambda_max": lmax, "E_star": E, "eps": 1e-10,
            "oracle": f"phase schedule, M={M}", "updates": r["n_updates"],
            "nnz": int(np.count_nonzero(r["Z"])), "input_sha256_16": input_hash(pb)}
        print(name, seed, res[f"{name}/seed{seed}"], f"{time.time() - t:.1f}s", flush=True)
    with open(OUT, "w") as f:
        json.dump(res, f, indent=1, sort_keys=True)


if __name__ == "__main__":
    main()
