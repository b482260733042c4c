"""The tensor-core (tcgen05) projection form against the FP32 CUDA-core form
and the oracle.

The FP16 hi/lo split product is exact to about 2^-22 relative, so away from
bucket boundaries it lands in the same bucket as the FP32 form; values
within 2^-11 of a boundary are recomputed by the FP32 form's arithmetic.
The keys of both forms must therefore be bit-identical, and both must match
the float64 oracle up to the boundary tolerance eta of test_gpu_parity.
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


def handle(mom, wl, precision, L, K, r, A, U):
    h = mom.Momenti(w=wl.w, d=wl.d, k=wl.k, delta=wl.delta, K=K, L=L, r=r, precision=precision)
    h.set_hash_params(A, U)
    h.hash_all(wl.series)
    return h


@pytest.mark.parametrize("case", ["plain_small", "plain_fp32_short", "ragged_f64"])
def test_tc_keys_equal_fp32_keys(mom, case):
    if case == "plain_small":
        wl, L, K = synth.plain_small(0), 16, 8
    elif case == "plain_fp32_short":
        wl, L, K = synth.plain_fp32(0, n=20_000), 40, 8
    else:
        wl, L, K = synth.tiny(31, n=1000, D=3, w=65, d=2, k=2, n_motifs=1), 37, 5
    A, U = synth.hash_draws(wl.D, L, K, wl.w, 9)
    r = O.estimate_r(wl.series, wl.w, A)
    h32 = handle(mom, wl, mom.PREC_FP32, L, K, r, A, U)
    htc = handle(mom, wl, mom.PREC_F16X2, L, K, r, A, U)
    _, st = htc.topk()
    assert st["precision_used"] == mom.PREC_F16X2
    M = wl.n - wl.w + 1
    assert st["n_rehashed"] <= 0.01 * M * wl.D * L * K + 100
    for j in range(L):
        np.testing.assert_array_equal(htc.keys(j), h32.keys(j), err_msg=f"repetition {j}")


def test_tc_topk_plain_small(mom):
    gold = json.load(open(os.path.join(GOLDEN, "exact_plain_small_seed0.json")))
    wl = synth.plain_small(0)
    h = mom.Momenti(w=wl.w, d=wl.d, k=wl.k, delta=wl.delta, precision=mom.PREC_F16X2)
    h.hash_all(wl.series)
    got, st = h.topk()
    assert st["precision_used"] == mom.PREC_F16X2
    assert [(m["a"], m["b"]) for m in got] == [(m[1], m[2]) for m in gold["motifs"]]
    for g, r in zip(got, gold["motifs"]):
        assert g["dist_d"] == pytest.approx(r[0], rel=1e-9)
        assert g["dims"] == tuple(r[3])
