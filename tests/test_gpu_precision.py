"""The precision form (D=32, w=500, d=8, k=10, delta=0.01, float32 series
of random walk, sinusoids and 5-sigma spikes, ten motifs planted in 8 dims)
through the C ABI.

* On its n = 2e5 prefix (the same generator at that length) the default
  search returns the exact top-k that tests/golden/make_golden.py wrote with
  the oracle's C pair enumeration: pairs and dims identical, distances
  within 1e-9 relative (float64 re-verification), in both projection forms.
* At full size (n = 1e6) the search returns the ten planted motifs, each
  re-verified in float64 against the oracle's own distance of that pair,
  and its float32 traversal error is stated.
"""
import json
import os

import numpy as np
import pytest

from oracle import momenti_oracle as O
from paper_2502_14446_gb300 import synth

pytestmark = pytest.mark.gpu
GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


@pytest.fixture(scope="module")
def mom():
    from paper_2502_14446_gb300 import build_ext
    build_ext.build()
    from paper_2502_14446_gb300 import momenti
    return momenti


@pytest.mark.parametrize("precision", ["f16x2", "fp32"])
def test_precision_prefix_matches_the_exact_top_k(mom, precision):
    gold = json.load(open(os.path.join(GOLDEN, "exact_precision_form_n200000_seed0.json")))
    wl = synth.precision_form(0, n=gold["n"])
    prec = mom.PREC_F16X2 if precision == "f16x2" else mom.PREC_FP32
    with mom.Momenti(w=wl.w, d=wl.d, k=wl.k, delta=wl.delta, precision=prec) as h:
        h.hash_all(wl.series)
        got, st = h.topk()
    ref = gold["motifs"]
    assert [(m["a"], m["b"]) for m in got] == [(m[1], m[2]) for m in ref]
    for g, r in zip(got, ref):
        assert g["dist_d"] == pytest.approx(r[0], rel=1e-9)
        assert g["dims"] == tuple(r[3])
        assert g["dist_max"] == pytest.approx(r[4], rel=1e-9)
    assert st["max_rel_err_fp32"] < 1e-4


def test_precision_full_size_returns_the_planted_motifs(mom):
    wl = synth.precision_form(0)
    with mom.Momenti(w=wl.w, d=wl.d, k=wl.k, delta=wl.delta) as h:
        h.hash_all(wl.series)
        got, st = h.topk()
    assert len(got) == wl.k
    planted = {(a, b): dims for a, b, dims in wl.planted}
    assert {(m["a"], m["b"]) for m in got} == set(planted)
    for m in got:
        dist = O.per_dim_distances(wl.series.astype(np.float64), wl.w, m["a"], m["b"])
        dd, dims, dmax = O.select_d(dist, wl.d)
        assert m["dist_d"] == pytest.approx(dd, rel=1e-9)
        assert m["dims"] == dims
        assert set(dims) == set(planted[(m["a"], m["b"])])
    assert st["max_rel_err_fp32"] < 1e-4
