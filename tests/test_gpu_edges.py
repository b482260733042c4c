"""Edge cases of the search through the C ABI: argument errors, one
dimension, all dimensions, fewer non-trivial motifs than k, constant
series, and repeated searches on one index.  Expected values come from the
oracle (oracle/momenti_oracle.py)."""
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


def pairs(motifs):
    return [(m["a"], m["b"]) for m in motifs]


def same(got, ref):
    assert pairs(got) == [(m[1], m[2]) for m in ref]
    for g, r in zip(got, ref):
        assert g["dims"] == tuple(r[3])
        assert g["dist_d"] == pytest.approx(r[0], rel=1e-9, abs=1e-9)


def test_argument_errors(mom):
    T = np.zeros((3, 50), np.float32)
    with mom.Momenti(w=60, d=1, k=1, delta=0.1) as h:     # series shorter than a window
        with pytest.raises(mom.MomentiError):
            h.hash_all(T)
    with mom.Momenti(w=10, d=4, k=1, delta=0.1) as h:     # d > D
        with pytest.raises(mom.MomentiError):
            h.hash_all(T)
    with mom.Momenti(w=10, d=1, k=1, delta=0.1) as h:     # more than 64 dims
        with pytest.raises(mom.MomentiError):
            h.hash_all(np.zeros((65, 50), np.float32))


@pytest.mark.parametrize("seed,D,d", [(31, 1, 1), (32, 3, 3)])
def test_one_dimension_and_all_dimensions(mom, seed, D, d):
    wl = synth.tiny(seed, 900, D, 30, d, k=3, n_motifs=1)
    ref = O.exact_topk(wl.series, wl.w, wl.d, wl.k)
    with mom.Momenti(w=wl.w, d=wl.d, k=wl.k, delta=wl.delta, precision=mom.PREC_FP32) as h:
        h.hash_all(wl.series)
        same(h.topk_exact(), ref)
        got, st = h.topk()
        if st["fallback"]:
            same(got, ref)


def test_fewer_motifs_than_k(mom):
    # n = 200, w = 40: windows more than 20 apart leave room for only a few
    # non-overlapping pairs, far fewer than k = 10
    wl = synth.tiny(33, 200, 2, 40, 1, k=10, n_motifs=0)
    with mom.Momenti(w=wl.w, d=wl.d, k=wl.k, delta=wl.delta, precision=mom.PREC_FP32) as h:
        h.hash_all(wl.series)
        got = h.topk_exact()
        got2, _ = h.topk()
    m = len(got)
    assert 0 < m < wl.k
    same(got, O.exact_topk(wl.series, wl.w, wl.d, m))
    assert O.exact_topk(wl.series, wl.w, wl.d, m + 1) is None
    assert pairs(got2) == pairs(got)


@pytest.mark.parametrize("dtype", [np.float32, np.float64])
def test_constant_series(mom, dtype):
    # every window is flat: every distance is 0, ties go to (a, b) order
    T = np.full((2, 400), 7.5, dtype=dtype)
    w, d, k = 40, 1, 3
    ref = O.exact_topk(T, w, d, k)
    with mom.Momenti(w=w, d=d, k=k, delta=0.1, precision=mom.PREC_FP32) as h:
        h.hash_all(T)
        got, _ = h.topk()
    assert pairs(got) == [(m[1], m[2]) for m in ref]
    assert all(m["dist_d"] == 0.0 for m in got)


def test_repeated_search_is_deterministic(mom):
    wl = synth.tiny(34, 3000, 4, 50, 2, k=4, n_motifs=2)
    with mom.Momenti(w=wl.w, d=wl.d, k=wl.k, delta=wl.delta) as h:
        h.hash_all(wl.series)
        a, sa = h.topk()
        b, sb = h.topk()
        h.hash_all(wl.series)
        c, sc = h.topk()
    assert a == b == c
    assert (sa["stop_i"], sa["stop_j"]) == (sb["stop_i"], sb["stop_j"]) == (sc["stop_i"], sc["stop_j"])
