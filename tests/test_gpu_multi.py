"""Motifs of several dimensionalities in one traversal (Section 6.3) on
the GPU, through momenti_topk_multi, against oracle.momenti_multi.

The device keys equal the oracle's except for hash values in the float32
band around a bucket edge (checked by the hash tests); the traversal is
compared unconditionally by running the oracle's loop on the device's own
keys: every d must be confirmed at the same (i, j), with the same TOP.
Top-k pairs and dims identical, distances within 1e-9 relative.
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


def same(got, ref, rel=1e-9):
    assert [(g["a"], g["b"]) for g in got] == [(x[1], x[2]) for x in ref]
    for g, x in zip(got, ref):
        assert g["dist_d"] == pytest.approx(x[0], rel=rel, abs=1e-9)
        assert g["dims"] == tuple(x[3])


@pytest.mark.parametrize("seed,D,d_low,d_high", [(1, 4, 1, 3), (2, 3, 1, 2), (3, 5, 2, 4)])
def test_multi_follows_the_oracle(mom, seed, D, d_low, d_high):
    wl = synth.tiny(seed, 1500, D, 50, d_high, k=2, n_motifs=2, noise=0.01)
    L, K, delta = 100, 8, 0.1
    A, U = synth.hash_draws(wl.D, L, K, wl.w, seed)
    r = O.estimate_r(wl.series, wl.w, A)
    h = mom.Momenti(w=wl.w, d=d_low, k=wl.k, delta=delta, K=K, L=L, r=r,
                    precision=mom.PREC_FP32, flags=mom.FLAG_NO_COST_SWITCH)
    h.set_hash_params(A, U)
    h.hash_all(wl.series)
    res, st = h.topk_multi(d_low, d_high)
    keys_dev = np.stack([h.keys(j) for j in range(L)])
    ref = O.momenti_multi(wl.series, wl.w, d_low, d_high, wl.k, delta, A, U, r, keys=keys_dev)
    for d in range(d_low, d_high + 1):
        motifs, stop = res[d]
        same(motifs, ref[d]["motifs"])
        assert stop == (ref[d]["stop"] or (0, 0)), d
        if ref[d]["stop"] is not None:
            assert motifs[-1]["fail_bound"] == pytest.approx(ref[d]["fail_bound"], rel=1e-3)
    # the oracle on its own keys returns the same motifs
    own = O.momenti_multi(wl.series, wl.w, d_low, d_high, wl.k, delta, A, U, r)
    for d in range(d_low, d_high + 1):
        same(res[d][0], own[d]["motifs"])
    h.close()


def test_multi_with_one_dimensionality_is_topk(mom):
    wl = synth.tiny(4, 1500, 3, 50, 2, k=2, n_motifs=2)
    for flags in (0, mom.FLAG_NO_COST_SWITCH):
        h = mom.Momenti(w=wl.w, d=2, k=wl.k, delta=wl.delta, L=100, precision=mom.PREC_FP32,
                        flags=flags)
        h.hash_all(wl.series)
        one, st1 = h.topk()
        res, st2 = h.topk_multi(2, 2)
        assert [(m["a"], m["b"], m["dims"]) for m in one] == \
            [(m["a"], m["b"], m["dims"]) for m in res[2][0]]
        assert (st1["stop_i"], st1["stop_j"]) == res[2][1] == (st2["stop_i"], st2["stop_j"])
        h.close()


def test_multi_each_d_is_the_exact_top_k(mom):
    # default search (cost switch on, device draws): every d's result is the
    # exact top-k of that d on this small, well-separated case
    wl = synth.tiny(5, 2000, 4, 50, 3, k=2, n_motifs=2, noise=0.01)
    with mom.Momenti(w=wl.w, d=1, k=wl.k, delta=0.05, precision=mom.PREC_F16X2) as h:
        h.hash_all(wl.series)
        res, st = h.topk_multi(1, 4)
    for d in range(1, 5):
        same(res[d][0], O.exact_topk(wl.series, wl.w, d, wl.k))


def test_multi_argument_errors(mom):
    wl = synth.tiny(6, 600, 3, 40, 1, k=1, n_motifs=0)
    with mom.Momenti(w=wl.w, d=1, k=1, delta=0.1, L=8) as h:
        h.hash_all(wl.series)
        for lo, hi in ((0, 2), (2, 1), (1, 4)):
            with pytest.raises(mom.MomentiError) as e:
                h.topk_multi(lo, hi)
            assert e.value.code == mom.ERR_ARG
