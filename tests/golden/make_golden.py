"""Writes the stored expected values of the parity tests.

Calls only the CPU oracle (oracle/momenti_oracle.py) on the seeded
synthetic inputs of paper_2502_14446_gb300.synth.  Each output file is a
small JSON record: the workload name and seed, the exact top-k motifs of
Definition (top-k multidimensional motifs, Section 3.1) as
[dist_d, a, b, dims, dist_max], and the oracle's wall time.

Usage: python tests/golden/make_golden.py plain_small plain_fp32 batch_small guarantee
       python tests/golden/make_golden.py precision_form large_form   (n = 2e5 prefixes)
       python tests/golden/make_golden.py stop   (Algorithm 1 stopped by STOP, full bench workload)

batch_small is the batching form at reduced lengths (6 series, n
log-uniform in [1500, 5000]); its file holds one record per series.
guarantee holds the exact top-2 of 100 small random-walk series (seeds
100..199: n=1500, D=3, w=50, d=2, two planted motifs) for the failure-rate
test of Lemma topk.
"""
import json
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import momenti_oracle as O  # noqa: E402
from paper_2502_14446_gb300 import synth  # noqa: E402

OUT = os.path.dirname(os.path.abspath(__file__))

# first threshold for the doubling search of exact_topk_auto; any value
# gives the same answer, a good one only saves passes
TAU0 = {"plain_small": None, "plain_fp32": 8.0}


def make(name: str, seed: int = 0):
    wl = getattr(synth, name)(seed)
    t0 = time.time()
    res = O.exact_topk_auto(wl.series, wl.w, wl.d, wl.k, tau0=TAU0.get(name), block=256)
    dt = time.time() - t0
    rec = {
        "workload": name, "seed": seed, "D": wl.D, "n": wl.n, "w": wl.w, "d": wl.d, "k": wl.k,
        "planted": [[a, b, list(dims)] for a, b, dims in wl.planted],
        "motifs": [[m[0], m[1], m[2], list(m[3]), m[4]] for m in res],
        "oracle_seconds": dt,
    }
    path = os.path.join(OUT, f"exact_{name}_seed{seed}.json")
    with open(path, "w") as fh:
        json.dump(rec, fh, indent=1)
    print(path, f"{dt:.1f}s")


def make_batch_small(seed: int = 0):
    wls = synth.batch_form(seed, count=6, n_lo=1500, n_hi=5000)
    recs = []
    t0 = time.time()
    for wl in wls:
        res = O.exact_topk(wl.series, wl.w, wl.d, wl.k, block=256)
        recs.append({
            "workload": wl.name, "D": wl.D, "n": wl.n, "w": wl.w, "d": wl.d, "k": wl.k,
            "planted": [[a, b, list(dims)] for a, b, dims in wl.planted],
            "motifs": [[m[0], m[1], m[2], list(m[3]), m[4]] for m in res],
        })
    dt = time.time() - t0
    path = os.path.join(OUT, f"exact_batch_small_seed{seed}.json")
    with open(path, "w") as fh:
        json.dump({"workload": "batch_small", "seed": seed, "series": recs,
                   "oracle_seconds": dt}, fh, indent=1)
    print(path, f"{dt:.1f}s")


def make_guarantee():
    recs = []
    t0 = time.time()
    for seed in range(100, 200):
        wl = synth.tiny(seed, 1500, 3, 50, 2, k=2, n_motifs=2)
        res = O.exact_topk(wl.series, wl.w, wl.d, wl.k, block=256)
        recs.append({"seed": seed, "motifs": [[m[0], m[1], m[2], list(m[3]), m[4]] for m in res]})
    dt = time.time() - t0
    path = os.path.join(OUT, "exact_guarantee_seeds100_199.json")
    with open(path, "w") as fh:
        json.dump({"workload": "tiny(seed, 1500, 3, 50, 2, k=2, n_motifs=2)", "series": recs,
                   "oracle_seconds": dt}, fh, indent=0)
    print(path, f"{dt:.1f}s")


# the larger forms at a length the oracle finishes in minutes (the same
# generator, its motifs planted inside that length), through the oracle's C
# pair enumeration (exact_topk_diag); first thresholds as above
PREFIX = {"precision_form": (200_000, 16.0), "large_form": (200_000, 40.0)}


def make_prefix(name: str, seed: int = 0):
    n, tau0 = PREFIX[name]
    wl = getattr(synth, name)(seed, n=n)
    t0 = time.time()
    res = O.exact_topk_diag(wl.series, wl.w, wl.d, wl.k, tau0=tau0)
    dt = time.time() - t0
    rec = {
        "workload": name, "seed": seed, "D": wl.D, "n": wl.n, "w": wl.w, "d": wl.d, "k": wl.k,
        "planted": [[a, b, list(dims)] for a, b, dims in wl.planted],
        "motifs": [[m[0], m[1], m[2], list(m[3]), m[4]] for m in res],
        "oracle": "exact_topk_diag", "oracle_seconds": dt, "host_threads": os.cpu_count(),
    }
    path = os.path.join(OUT, f"exact_{name}_n{n}_seed{seed}.json")
    with open(path, "w") as fh:
        json.dump(rec, fh, indent=1)
    print(path, f"{dt:.1f}s")


# Algorithm 1 stopped by Algorithm 2 on the full bench workload: the
# plain float32 form (D=8, n=1e5, w=300, d=3, delta=0.05) asked for its
# k = 5 closest motifs, with the fixed width r = 8 of the paper's r
# experiment and the seed-0 hash draws (K=8, L=200) that the GPU test sets
# through set_hash_params; the oracle's hashing and traversal in the
# paper's loop order, no exact fallback
STOP = {"k": 5, "r": 8.0, "L": 200, "K": 8}


def make_stop(seed: int = 0):
    wl = synth.plain_fp32(seed)
    T = wl.series.astype("float64")
    A, U = synth.hash_draws(wl.D, STOP["L"], STOP["K"], wl.w, seed)
    t0 = time.time()
    keys, _ = O.hash_all(T, wl.w, A, U, STOP["r"])
    Z = [O.znorm_windows(T[f], wl.w) for f in range(wl.D)]
    top, stop, n_dist, _ = O.momenti_traverse(keys, lambda a, b: O._pair_distances(Z, a, b),
                                              wl.d, STOP["k"], wl.delta, STOP["r"],
                                              O.exclusion_zone(wl.w), STOP["K"])
    dt = time.time() - t0
    rec = {
        "workload": "plain_fp32", "seed": seed, "D": wl.D, "n": wl.n, "w": wl.w, "d": wl.d,
        "delta": wl.delta, **STOP, "hash_seed": seed,
        "stop": list(stop) if stop else None, "n_dist": n_dist,
        "fail_bound": (O.failure_bound(top[-1][4], stop[0], stop[1], STOP["K"], STOP["L"], wl.d,
                                       STOP["r"]) if stop else None),
        "motifs": [[m[0], m[1], m[2], list(m[3]), m[4]] for m in top],
        "oracle": "hash_all + momenti_traverse", "oracle_seconds": dt,
    }
    path = os.path.join(OUT, f"stop_plain_fp32_k{STOP['k']}_r{int(STOP['r'])}_seed{seed}.json")
    with open(path, "w") as fh:
        json.dump(rec, fh, indent=1)
    print(path, f"{dt:.1f}s")


if __name__ == "__main__":
    for nm in sys.argv[1:] or ["plain_small"]:
        if nm == "batch_small":
            make_batch_small()
        elif nm == "guarantee":
            make_guarantee()
        elif nm in PREFIX:
            make_prefix(nm)
        elif nm == "stop":
            make_stop()
        else:
            make(nm)
