"""Write the stored reference values of the benchmark workloads.

Calls only the FP64 oracle (oracle/) on inputs from the seeded generator:
for each (workload, seed) it records lambda = 0.1 * lambda_max, the optimum
E* = E(Z*) reached by the oracle's phase-schedule locally greedy CD at
eps = 1e-10, and a hash of the generated inputs so a reader can tell when
the generator no longer reproduces them.

    python tests/golden/make_golden.py            # all single-signal entries
    python tests/golden/make_golden.py --batch    # the 512-signal batch (8 processes)
    python tests/golden/make_golden.py --verylong # the T = 5e6 recording, with Z*
    python tests/golden/make_golden.py --image2d  # the 512 x 512 image (2-D oracle)

The very long recording's entry (about 7 minutes of oracle time) also stores
the oracle's sparse Z* (verylong_seed0_zstar.npz: flat indices k * Tz + t of
the nonzeros, ascending, and their values rounded to float32, a relative
2^-24 that is far below the 1e-4 comparison bar), so that a GPU solve at full
size can be compared coordinate by coordinate.

The batch entries (optimum_batch.json) hold, per signal of the batch
workload, lambda_i = 0.1 * lambda_max_i and E*_i, plus one hash over all
signals' inputs.
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


OUT_BATCH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "optimum_batch.json")
BATCH = ("batch_P7_K25_L64_n512_T10000_500000", 0)


def _batch_entry(i):
    name, seed = BATCH
    T = synth.batch_lengths(synth.BATCH_WORKLOADS[name]["n"],
                            synth.BATCH_WORKLOADS[name]["T_min"],
                            synth.BATCH_WORKLOADS[name]["T_max"], seed)
    pb = synth.batch_signal(name, seed, i, int(T[i]))
    lmax = oracle.lambda_max(pb.D, pb.X)
    lam = 0.1 * lmax
    M = max(1, pb.Tz // (2 * pb.L - 2))
    r = oracle.locally_greedy_cd(pb.D, pb.X, lam, 1e-10, M=M, mode="phase")
    assert r["converged"]
    E = oracle.objective(pb.D, pb.X, r["Z"], lam)
    h = hashlib.sha256()
    h.update(pb.X.tobytes())
    return {"i": i, "T": int(T[i]), "lambda": lam, "lambda_max": lmax, "E_star": E,
            "updates": r["n_updates"], "nnz": int(np.count_nonzero(r["Z"])),
            "x_sha256": h.hexdigest()}


def batch_hash(D, x_hashes) -> str:
    h = hashlib.sha256()
    h.update(D.tobytes())
    for x in x_hashes:
        h.update(x.encode())
    return h.hexdigest()[:16]


def main_batch(workers: int = 8):
    import multiprocessing as mp
    name, seed = BATCH
    n = synth.BATCH_WORKLOADS[name]["n"]
    t = time.time()
    # longest first so the pool's tail is short
    T = synth.batch_lengths(n, synth.BATCH_WORKLOADS[name]["T_min"],
                            synth.BATCH_WORKLOADS[name]["T_max"], seed)
    order = [int(i) for i in np.argsort(-T)]
    with mp.get_context("spawn").Pool(workers) as pool:
        rows = {}
        for r in pool.imap_unordered(_batch_entry, order):
            rows[r["i"]] = r
            if len(rows) % 32 == 0:
                print(f"{len(rows)}/{n} {time.time() - t:.0f}s", flush=True)
    rows = [rows[i] for i in range(n)]
    D = synth.make_dictionary(synth.BATCH_WORKLOADS[name]["K"], synth.BATCH_WORKLOADS[name]["P"],
                              synth.BATCH_WORKLOADS[name]["L"], seed)
    out = {"workload": name, "seed": seed, "eps": 1e-10,
           "oracle": "phase schedule, M = max(1, floor(Tz / (2L - 2))) per signal",
           "input_sha256_16": batch_hash(D, [r["x_sha256"] for r in rows]),
           "T": [r["T"] for r in rows], "lambda": [r["lambda"] for r in rows],
           "lambda_max": [r["lambda_max"] for r in rows], "E_star": [r["E_star"] for r in rows],
           "updates": [r["updates"] for r in rows], "nnz": [r["nnz"] for r in rows]}
    with open(OUT_BATCH, "w") as f:
        json.dump(out, f, indent=0)
    print(f"done in {time.time() - t:.0f}s", flush=True)


VERYLONG = ("verylong_P1_K25_L200_T5000000", 0)
OUT_ZSTAR = os.path.join(os.path.dirname(os.path.abspath(__file__)), "verylong_seed0_zstar.npz")


def main_verylong():
    name, seed = VERYLONG
    t = time.time()
    pb = synth.make_workload(name, seed=seed)
    lmax = oracle.lambda_max(pb.D, pb.X)
    lam = 0.1 * lmax
    M = pb.Tz // (2 * pb.L - 2)
    r = oracle.locally_greedy_cd(pb.D, pb.X, lam, 1e-10, M=M, mode="phase")
    assert r["converged"]
    E = oracle.objective(pb.D, pb.X, r["Z"], lam)
    flat = np.flatnonzero(r["Z"])
    np.savez_compressed(OUT_ZSTAR, index=flat.astype(np.int64),
                        value=r["Z"].reshape(-1)[flat].astype(np.float32),
                        shape=np.array(r["Z"].shape, np.int64))
    with open(OUT) as f:
        res = json.load(f)
    res[f"{name}/seed{seed}"] = {
        "lambda": lam, "lambda_max": lmax, "E_star": E, "eps": 1e-10,
        "oracle": f"phase schedule, M={M}", "updates": r["n_updates"],
        "nnz": int(flat.size), "zinf": float(np.abs(r["Z"]).max()),
        "input_sha256_16": input_hash(pb), "zstar": os.path.basename(OUT_ZSTAR)}
    with open(OUT, "w") as f:
        json.dump(res, f, indent=1, sort_keys=True)
    print(name, seed, res[f"{name}/seed{seed}"], f"{time.time() - t:.1f}s", flush=True)


IMAGE = ("image_P1_K8_h8_w8_512x512", 0)


def main_image2d():
    from oracle import csc2d
    name, seed = IMAGE
    t = time.time()
    pb = synth.make_image_workload(name, seed=seed)
    lmax = csc2d.lambda_max(pb.D, pb.X)
    lam = 0.1 * lmax
    Hz = pb.X.shape[1] - pb.D.shape[2] + 1
    M = max(1, Hz // (2 * pb.D.shape[2] - 2))
    r = csc2d.locally_greedy_cd(pb.D, pb.X, lam, 1e-10, M=M, mode="phase")
    assert r["converged"]
    E = csc2d.objective(pb.D, pb.X, r["Z"], lam)
    with open(OUT) as f:
        res = json.load(f)
    res[f"{name}/seed{seed}"] = {
        "lambda": lam, "lambda_max": lmax, "E_star": E, "eps": 1e-10,
        "oracle": f"band phase schedule, M={M}", "updates": r["n_updates"],
        "nnz": int(np.count_nonzero(r["Z"])), "input_sha256_16": input_hash(pb)}
    with open(OUT, "w") as f:
        json.dump(res, f, indent=1, sort_keys=True)
    print(name, seed, res[f"{name}/seed{seed}"], f"{time.time() - t:.1f}s", flush=True)


def main():
    if "--batch" in sys.argv[1:]:
        return main_batch()
    if "--image2d" in sys.argv[1:]:
        return main_image2d()
    if "--verylong" in sys.argv[1:]:
        return main_verylong()
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
    try:
        with open(OUT) as f:
            old = json.load(f)
        res.update({k: v for k, v in old.items()
                    if k.startswith(VERYLONG[0]) or k.startswith(IMAGE[0])})
    except (OSError, ValueError):
        pass
    with open(OUT, "w") as f:
        json.dump(res, f, indent=1, sort_keys=True)


if __name__ == "__main__":
    main()
