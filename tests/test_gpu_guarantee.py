"""Failure rate of the top-k across seeds (Lemma topk): every returned motif
is the true one with probability at least 1 - delta.

100 small random-walk series with two planted motifs (seeds 100..199:
n=1500, D=3, w=50, d=2, k=2, delta=0.1), searched through Algorithm 1's
loop without the cost switch, so that STOP decides where it can; the exact
top-k of each series comes from tests/golden/exact_guarantee_seeds100_199.json
(written by tests/golden/make_golden.py from the oracle only).

A motif misses when the pair at its rank differs from the exact one.  The
misses over the 200 (series, rank) trials must stay within the one-sided
99% quantile of Binomial(200, delta); the test also requires STOP to hold
on a fair share of the series, so that the probabilistic branch is the one
being tested (the exact branch never misses).
"""
import json
import math
import os

import pytest

from paper_2502_14446_gb300 import synth

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden",
                      "exact_guarantee_seeds100_199.json")


@pytest.fixture(scope="module")
def mom():
    from paper_2502_14446_gb300 import build_ext
    build_ext.build()
    from paper_2502_14446_gb300 import momenti
    return momenti


def binom_quantile(n, p, q):
    """Smallest x with P(X <= x) >= q for X ~ Binomial(n, p)."""
    c = 0.0
    for x in range(n + 1):
        c += math.comb(n, x) * p ** x * (1 - p) ** (n - x)
        if c >= q:
            return x
    return n


def test_failure_rate_within_delta(mom):
    gold = json.load(open(GOLDEN))
    misses = trials = stopped = 0
    for rec in gold["series"]:
        wl = synth.tiny(rec["seed"], 1500, 3, 50, 2, k=2, n_motifs=2)
        with mom.Momenti(w=wl.w, d=wl.d, k=wl.k, delta=wl.delta, precision=mom.PREC_FP32,
                         flags=mom.FLAG_NO_COST_SWITCH) as h:
            h.hash_all(wl.series)
            got, st = h.topk()
        stopped += st["stop_i"] > 0
        exact = [(m[1], m[2]) for m in rec["motifs"]]
        for q, pair in enumerate(exact):
            trials += 1
            misses += q >= len(got) or (got[q]["a"], got[q]["b"]) != pair
    bound = binom_quantile(trials, wl.delta, 0.99)
    assert stopped >= 25, f"STOP held on only {stopped} series"
    assert misses <= bound, f"{misses} misses in {trials} trials (bound {bound})"
