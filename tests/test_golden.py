"""The stored expected values (tests/golden/) are what the committed oracle
computes: the small files' records are recomputed on the CPU from the same
seeded inputs (same pairs and dims, distances to 1e-9)."""
import json
import os

import pytest

from oracle import momenti_oracle as O
from paper_2502_14446_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def same(motifs, stored):
    assert [(m[1], m[2], tuple(m[3])) for m in motifs] == [(s[1], s[2], tuple(s[3])) for s in stored]
    for m, s in zip(motifs, stored):
        assert m[0] == pytest.approx(s[0], rel=1e-9, abs=1e-12)
        assert m[4] == pytest.approx(s[4], rel=1e-9, abs=1e-12)


def test_plain_small_golden_is_the_oracles():
    rec = json.load(open(os.path.join(GOLDEN, "exact_plain_small_seed0.json")))
    wl = synth.plain_small(rec["seed"])
    assert (wl.D, wl.n, wl.w, wl.d, wl.k) == (rec["D"], rec["n"], rec["w"], rec["d"], rec["k"])
    assert [[a, b, list(dims)] for a, b, dims in wl.planted] == rec["planted"]
    same(O.exact_topk_auto(wl.series, wl.w, wl.d, wl.k, block=256), rec["motifs"])


def test_guarantee_golden_is_the_oracles():
    rec = json.load(open(os.path.join(GOLDEN, "exact_guarantee_seeds100_199.json")))
    for s in rec["series"][:5]:
        wl = synth.tiny(s["seed"], 1500, 3, 50, 2, k=2, n_motifs=2)
        same(O.exact_topk(wl.series, wl.w, wl.d, wl.k, block=256), s["motifs"])


def test_stop_golden_is_consistent():
    # the full-size STOP record: its TOP is the stored exact top-5 of the
    # same workload (distances by the definition, to 1e-9), each motif's
    # distances re-evaluated here, and its bound is Lemma stop's at the
    # recorded (i, j) for the k-th's dist_max, at most delta
    rec = json.load(open(os.path.join(GOLDEN, "stop_plain_fp32_k5_r8_seed0.json")))
    exact = json.load(open(os.path.join(GOLDEN, "exact_plain_fp32_seed0.json")))["motifs"]
    same(rec["motifs"], exact[:rec["k"]])
    wl = synth.plain_fp32(rec["seed"])
    T = wl.series.astype("float64")
    for m in rec["motifs"]:
        dd, dims, dmax = O.select_d(O.per_dim_distances(T, wl.w, m[1], m[2]), wl.d)
        assert dd == pytest.approx(m[0], rel=1e-9) and list(dims) == m[3]
        assert dmax == pytest.approx(m[4], rel=1e-9)
    i, j = rec["stop"]
    fb = O.failure_bound(rec["motifs"][-1][4], i, j, rec["K"], rec["L"], rec["d"], rec["r"])
    assert fb == pytest.approx(rec["fail_bound"], rel=1e-12) and fb <= rec["delta"]
    # one repetition earlier the bound is still above delta, so (i, j) is
    # the first point where STOP can hold with this TOP
    assert O.failure_bound(rec["motifs"][-1][4], i, j - 1, rec["K"], rec["L"], rec["d"],
                           rec["r"]) > rec["delta"]
