"""The anytime search (Section 4, the remark after Algorithm 1) through
momenti_search_begin / step / current / finish.

TOP only admits better pairs, so the k-th distance of the current TOP never
grows while the search advances; each current candidate's miss bound is
Lemma stop's bound (the oracle's failure_bound) for its own dist_d^max
after the repetitions processed so far; stepping and finishing gives the
result and stopping point of one momenti_topk call.  Distances of the
intermediate TOP are the traversal's float32 form (1e-4 relative of the
oracle's float64 distance), the final ones float64 (1e-9).
"""
import numpy as np
import pytest

from oracle import momenti_oracle as O
from paper_2502_14446_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mom():
    from paper_2502_14446_gb300 import build_ext
    build_ext.build()
    from paper_2502_14446_gb300 import momenti
    return momenti


@pytest.mark.parametrize("seed,flags_name", [(1, "NO_COST_SWITCH"), (2, "NO_COST_SWITCH"),
                                             (3, "default")])
def test_stepping_gives_the_result_of_topk(mom, seed, flags_name):
    wl = synth.tiny(seed, 1500, 3, 50, 2, k=2, n_motifs=2)
    flags = mom.FLAG_NO_COST_SWITCH if flags_name == "NO_COST_SWITCH" else 0
    kw = dict(w=wl.w, d=wl.d, k=wl.k, delta=wl.delta, L=100, precision=mom.PREC_FP32,
              flags=flags)
    with mom.Momenti(**kw) as h:
        h.hash_all(wl.series)
        ref, st_ref = h.topk()
        r = h.info()["r"]
        K, L = 8, h.info()["L"]
        h.search_begin()
        kths, steps = [], 0
        Z = [O.znorm_windows(wl.series[f], wl.w) for f in range(wl.D)]
        while not h.search_step(7):
            steps += 1
            cur, (i, j, ended) = h.search_current()
            top = cur[wl.d]
            assert 1 <= i <= K and 1 <= j <= L and not ended
            if len(top) == wl.k:
                kths.append(top[-1]["dist_d"])
            for m in top:
                # the candidate's own distance and its miss bound at (i, j)
                dist = O.per_dim_distances(wl.series, wl.w, m["a"], m["b"])
                dd, dims, dmax = O.select_d(dist, wl.d)
                assert m["dist_d"] == pytest.approx(dd, rel=1e-4, abs=1e-4)
                exp = O.failure_bound(m["dist_max"], i, j, K, L, wl.d, r)
                assert m["fail_bound"] == pytest.approx(exp, rel=1e-9, abs=1e-12)
        assert steps >= 1
        assert all(x >= y - 1e-6 for x, y in zip(kths, kths[1:]))      # only better pairs enter
        res, st = h.search_finish()
        got, stop = res[wl.d]
        assert [(m["a"], m["b"], m["dims"]) for m in got] == \
            [(m["a"], m["b"], m["dims"]) for m in ref]
        for g, x in zip(got, ref):
            assert g["dist_d"] == pytest.approx(x["dist_d"], rel=1e-9)
        assert stop == (st_ref["stop_i"], st_ref["stop_j"])
        assert st["fallback"] == st_ref["fallback"]


def test_search_calls_out_of_order(mom):
    wl = synth.tiny(4, 800, 2, 40, 1, k=1, n_motifs=1)
    with mom.Momenti(w=wl.w, d=1, k=1, delta=0.1, L=16) as h:
        with pytest.raises(mom.MomentiError) as e:
            h.search_step(1)
        assert e.value.code == mom.ERR_STATE          # no index, no search
        h.hash_all(wl.series)
        with pytest.raises(mom.MomentiError) as e:
            h.search_step(1)
        assert e.value.code == mom.ERR_STATE          # no search begun
        h.search_begin()
        h.search_step(3)
        h.hash_all(wl.series)                         # a new index ends the search
        with pytest.raises(mom.MomentiError) as e:
            h.search_current()
        assert e.value.code == mom.ERR_STATE
        h.search_begin()
        with pytest.raises(mom.MomentiError) as e:
            h.search_step(0)
        assert e.value.code == mom.ERR_ARG
        res, st = h.search_finish()
        ex = O.exact_topk(wl.series, wl.w, 1, 1)
        if st["fallback"]:
            assert [(m["a"], m["b"]) for m in res[1][0]] == [(x[1], x[2]) for x in ex]
