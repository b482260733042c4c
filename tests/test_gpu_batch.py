"""Batching form: many independent series of uneven length, dimension count
and window length searched at once through momenti_topk_batch.

Batching changes only the schedule (worker handles on their own streams and
host threads, longest series first), not the arithmetic: every series must give the motifs the
exact oracle gives (tests/golden/exact_batch_small_seed0.json, written by
tests/golden/make_golden.py from oracle/ only), with pairs and dimension
sets identical and distances within 1e-9 relative (the result is
re-verified in float64), and the same motifs as a one-at-a-time search of
the same handle parameters.
"""
import json
import os

import numpy as np
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


def _same(got, ref):
    assert len(got) == len(ref)
    for g, r in zip(got, ref):
        assert (g["a"], g["b"]) == (r[1], r[2])
        assert g["dims"] == tuple(r[3])
        assert g["dist_d"] == pytest.approx(r[0], rel=1e-9, abs=1e-9)


def _params(wls, precision):
    return [dict(w=wl.w, d=wl.d, k=wl.k, delta=wl.delta, precision=precision) for wl in wls]


@pytest.mark.parametrize("precision", ["fp32", "f16x2"])
def test_batch_matches_exact_oracle(mom, precision):
    gold = json.load(open(os.path.join(GOLDEN, "exact_batch_small_seed0.json")))
    wls = synth.batch_form(gold["seed"], count=len(gold["series"]), n_lo=1500, n_hi=5000)
    prec = mom.PREC_FP32 if precision == "fp32" else mom.PREC_F16X2
    res = mom.topk_batch(_params(wls, prec), [wl.series for wl in wls], threads=4)
    for (motifs, st), rec, wl in zip(res, gold["series"], wls):
        assert (rec["D"], rec["n"], rec["w"]) == (wl.D, wl.n, wl.w)
        _same(motifs, rec["motifs"])
        assert st["n_windows"] == wl.n - wl.w + 1


def test_batch_equals_one_at_a_time(mom):
    wls = synth.batch_form(1, count=5, n_lo=1500, n_hi=4000)
    batched = mom.topk_batch(_params(wls, mom.PREC_FP32), [wl.series for wl in wls], threads=3)
    for (motifs, st), wl in zip(batched, wls):
        with mom.Momenti(w=wl.w, d=wl.d, k=wl.k, delta=wl.delta, precision=mom.PREC_FP32) as h1:
            h1.hash_all(wl.series)
            one, st1 = h1.topk()
        assert [(m["a"], m["b"], m["dims"]) for m in motifs] == \
            [(m["a"], m["b"], m["dims"]) for m in one]
        assert [m["dist_d"] for m in motifs] == pytest.approx([m["dist_d"] for m in one],
                                                              rel=1e-12)
        assert (st["L"], st["K"], st["r"]) == (st1["L"], st1["K"], st1["r"])


def test_batch_device_series_and_errors(mom):
    torch = pytest.importorskip("torch")
    wls = synth.batch_form(2, count=3, n_lo=1200, n_hi=2500)
    ps = _params(wls, mom.PREC_FP32)
    dev = [torch.from_numpy(wl.series).cuda() for wl in wls]
    torch.cuda.synchronize()
    from_dev = mom.topk_batch(ps, dev, threads=2)
    from_host = mom.topk_batch(ps, [wl.series for wl in wls], threads=2)
    for (m0, _), (m1, _) in zip(from_dev, from_host):
        assert [(m["a"], m["b"], m["dims"]) for m in m0] == \
            [(m["a"], m["b"], m["dims"]) for m in m1]
    # a series shorter than its window fails alone and is named
    bad = np.zeros((3, wls[1].w - 1), np.float32)
    with pytest.raises(mom.MomentiError, match="series 1"):
        mom.topk_batch(ps[:2], [wls[0].series, bad], threads=2)
    # invalid parameters fail that series only
    with pytest.raises(mom.MomentiError, match="series 0"):
        mom.topk_batch([dict(ps[0], d=0), ps[1]], [wls[0].series, wls[1].series])
    # an empty batch is a no-op
    assert mom.topk_batch([], []) == []
