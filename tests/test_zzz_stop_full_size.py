"""Algorithm 1 stopped by Algorithm 2 at full size, through the C ABI.

The bench workload (plain float32 form: D=8, n=1e5, w=300, d=3,
delta=0.05), asked for its k = 5 closest motifs with the fixed width r = 8
(a value of the paper's r experiment), the seed-0 hash draws (K=8, L=200)
and the printed loop (no cost switch).  tests/golden/make_golden.py ran the
oracle's hashing and traversal on the same draws: STOP holds at level 8
and TOP is then the workload's exact top-5, the first five motifs of
tests/golden/exact_plain_fp32_seed0.json.  The device must stop by
Algorithm 2, with and without the cost switch, at the oracle's level and,
within a few repetitions, at its j
(a hash value in the float32 band around a bucket edge can move a
collision by a repetition), return the same five motifs with their float64
distances and dims, and report a miss bound of at most delta for the k-th.
"""
import json
import os

import pytest

from paper_2502_14446_gb300 import synth

pytestmark = pytest.mark.gpu
GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


@pytest.fixture(scope="module")
def mom():
    from paper_2502_14446_gb300 import build_ext
    build_ext.build()
    from paper_2502_14446_gb300 import momenti
    return momenti


@pytest.mark.parametrize("cost_switch", [False, True])
def test_full_size_search_stops_by_algorithm_2(mom, cost_switch):
    # with the cost switch on (the default) the search must still stop by
    # Algorithm 2: the level-8 probe predicts almost no traversal work, so
    # the switch does not abandon a search that stops cheaply
    gold = json.load(open(os.path.join(GOLDEN, "stop_plain_fp32_k5_r8_seed0.json")))
    exact = json.load(open(os.path.join(GOLDEN, "exact_plain_fp32_seed0.json")))["motifs"]
    exact = exact[:gold["k"]]
    # the oracle's own run stopped, and at the exact top-k
    assert gold["stop"] is not None and gold["fail_bound"] <= gold["delta"]
    assert [(m[1], m[2]) for m in gold["motifs"]] == [(m[1], m[2]) for m in exact]
    wl = synth.plain_fp32(0)
    A, U = synth.hash_draws(wl.D, gold["L"], gold["K"], wl.w, gold["hash_seed"])
    with mom.Momenti(w=wl.w, d=wl.d, k=gold["k"], delta=wl.delta, K=gold["K"], L=gold["L"],
                     r=gold["r"], precision=mom.PREC_FP32,
                     flags=0 if cost_switch else mom.FLAG_NO_COST_SWITCH,
                     mem_limit=wl.mem_limit) as h:
        h.set_hash_params(A, U)
        h.hash_all(wl.series)
        got, st = h.topk()
    assert st["fallback"] == 0 and st["switch_level"] == 0
    assert st["stop_i"] == gold["stop"][0]
    assert abs(st["stop_j"] - gold["stop"][1]) <= 5
    assert [(m["a"], m["b"]) for m in got] == [(m[1], m[2]) for m in exact]
    for g, r in zip(got, exact):
        assert g["dist_d"] == pytest.approx(r[0], rel=1e-9)
        assert g["dims"] == tuple(r[3])
    assert got[-1]["fail_bound"] <= wl.delta
