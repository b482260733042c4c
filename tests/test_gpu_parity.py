"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

Every test here runs on a GB300.  Inputs are the seeded synthetic series of
paper_2502_14446_gb300.synth; expected values come from oracle/ (or from
tests/golden/, written by tests/golden/make_golden.py, which calls only the
oracle).

Tolerances:
* window statistics: float64 running sums vs the two-pass oracle,
  relative 1e-10;
* hash values: bit-exact, except a value whose exact (a . z + b) / r lies
  within eta of an integer, where the float32 evaluation may land on either
  side; eta is the forward error bound of the float32 formula,
  ((w + 8) u sum_t |a_t z_t| + 4 u |a . z + b|) / r + 4 u |t|, u = 2^-24,
  doubled; those values may differ by one bucket;
* distances: float32 form within 1e-4 relative (+1e-4 absolute) of
  float64; float64 form within 1e-9 relative;
* top-k: motif pairs and dimension sets identical, distances within 1e-9
  relative (the result is re-verified in float64).
"""
import json
import math
import os

import numpy as np
import pytest

from oracle import momenti_oracle as O
from paper_2502_14446_gb300 import synth

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
U32 = 2.0 ** -24


@pytest.fixture(scope="module")
def mom():
    from paper_2502_14446_gb300 import build_ext
    build_ext.build()
    from paper_2502_14446_gb300 import momenti
    return momenti


def make(mom, wl, L=16, K=8, r=0.0, hash_seed=0, explicit=True, precision=None, **kw):
    prec = mom.PREC_FP32 if precision is None else precision
    h = mom.Momenti(w=wl.w, d=wl.d, k=wl.k, delta=wl.delta, K=K, L=L, r=r,
                    precision=prec, **kw)
    A = U = None
    if explicit:
        A, U = synth.hash_draws(wl.D, L, K, wl.w, hash_seed)
        h.set_hash_params(A, U)
    h.hash_all(wl.series)
    return h, A, U


def hash_tolerance(T, w, A, U, r, f):
    """eta of the module docstring for every (window, j, k) of dim f."""
    Z = O.znorm_windows(T[f], w)
    L, K = A.shape[1], A.shape[2]
    absdot = np.abs(Z) @ np.abs(A[f].astype(np.float64)).reshape(-1, w).T
    v = Z @ A[f].astype(np.float64).reshape(-1, w).T
    b = (U[f].astype(np.float64) * r).reshape(-1)
    t = (v + b) / r
    eta = ((w + 8) * U32 * absdot + 4 * U32 * np.abs(v + b)) / r + 4 * U32 * np.abs(t)
    return (2 * eta).reshape(-1, L, K)


def key_bytes(keys):
    return np.stack([(keys >> np.uint64(56 - 8 * k)) & np.uint64(255) for k in range(8)], -1).astype(np.int16)


# ------------------------------------------------------------ statistics

@pytest.mark.parametrize("case", ["f64", "f32"])
def test_window_stats(mom, case):
    if case == "f64":
        wl = synth.plain_small(0)
    else:
        wl = synth.plain_fp32(0, n=20_000)
    h, _, _ = make(mom, wl, L=2)
    mu, sd = h.window_stats()
    for f in range(wl.D):
        m0, s0, _ = O.window_stats(wl.series[f], wl.w)
        np.testing.assert_allclose(mu[f], m0, rtol=1e-10, atol=1e-10 * np.abs(m0).max())
        np.testing.assert_allclose(sd[f], s0, rtol=1e-10)


def test_flat_windows_and_short_series(mom):
    wl = synth.tiny(11, n=600, D=2, w=40, d=1, k=2, n_motifs=1)
    T = wl.series.copy()
    T[1, 100:260] = 3.25                       # flat run: windows 100..220 flat
    wl.series = T
    h, _, _ = make(mom, wl, L=4)
    mu, sd = h.window_stats()
    _, _, flat = O.window_stats(T[1], 40)
    assert (sd[1][flat] <= 1e-8 * (1 + np.abs(mu[1][flat]))).all()
    pairs = [(100, 200), (100, 300), (5, 300), (150, 400)]
    per, _, _ = h.verify(pairs, fp64=True)
    for q, (a, b) in enumerate(pairs):
        np.testing.assert_allclose(per[q], O.per_dim_distances(T, 40, a, b), rtol=1e-9, atol=1e-9)
    assert per[0, 1] == 0.0                    # flat vs flat
    assert per[1, 1] == pytest.approx(math.sqrt(40), rel=1e-12)
    # n == w: a single window, no pair at all
    one = synth.tiny(12, n=40, D=2, w=40, d=1, k=1, n_motifs=0)
    h1, _, _ = make(mom, one, L=2)
    motifs, _ = h1.topk()
    assert motifs == []


# --------------------------------------------------------------- hashes

@pytest.mark.parametrize("precision", ["fp32"])
def test_hash_keys_match_oracle(mom, precision):
    wl = synth.plain_small(0)
    L = 16
    A, U = synth.hash_draws(wl.D, L, 8, wl.w, 3)
    r = O.estimate_r(wl.series, wl.w, A)
    h, _, _ = make(mom, wl, L=L, r=r, hash_seed=3)
    assert h.info()["r"] == r
    keys_o, ts = O.hash_all(wl.series, wl.w, A, U, r)
    ho = np.clip(np.floor(ts), -128, 127)                   # (D, M, L, K)
    amb_total = diff_total = 0
    for j in range(L):
        kg = key_bytes(h.keys(j)) - 128                      # (M, D, 8)
        for f in range(wl.D):
            eta = hash_tolerance(wl.series, wl.w, A, U, r, f)[:, j, :]
            t = ts[f, :, j, :]
            amb = np.abs(t - np.round(t)) <= eta
            g = kg[:, f, :]
            o = ho[f, :, j, :]
            assert (g[~amb] == o[~amb]).all()
            assert (np.abs(g[amb] - o[amb]) <= 1).all()
            amb_total += int(amb.sum())
            diff_total += int((g != o).sum())
    # the band is about 2 eta wide; actual float32 errors are far below eta
    assert amb_total <= 0.02 * ts.size
    assert diff_total <= 1e-4 * ts.size


def test_r_heuristic_matches_oracle(mom):
    wl = synth.plain_small(0)
    L = 4
    A, U = synth.hash_draws(wl.D, L, 8, wl.w, 5)
    h, _, _ = make(mom, wl, L=L, hash_seed=5)
    r_o = O.estimate_r(wl.series, wl.w, A)
    assert h.info()["r"] == pytest.approx(r_o, rel=2e-5)


# --------------------------------------------------------------- index

def agreeing_segments(h, wl, A, U, r, L):
    keys_o, _ = O.hash_all(wl.series, wl.w, A, U, r)
    ok = np.zeros((L, wl.D), dtype=bool)
    for j in range(L):
        kg = h.keys(j)
        ok[j] = (kg == keys_o[j]).all(axis=0)
    return keys_o, ok


@pytest.mark.parametrize("n,D,L,r_scale", [(3000, 3, 6, 1.0), (6000, 2, 3, 40.0),
                                           (12000, 2, 2, 400.0)])
def test_index_matches_oracle(mom, n, D, L, r_scale):
    # r_scale widens the buckets (long runs of equal hash values)
    wl = synth.tiny(21, n=n, D=D, w=64, d=2, k=2, n_motifs=1)
    A, U = synth.hash_draws(wl.D, L, 8, wl.w, 21)
    r = O.estimate_r(wl.series, wl.w, A) * r_scale
    h, _, _ = make(mom, wl, L=L, r=r, hash_seed=21)
    keys_o, ok = agreeing_segments(h, wl, A, U, r, L)
    assert ok.mean() > 0.5
    order_o, lcp_o = O.build_index(keys_o)
    checked = 0
    for j in range(L):
        for f in range(wl.D):
            if not ok[j, f]:
                continue
            og, lg = h.index(j, f)
            np.testing.assert_array_equal(og, order_o[j, f])
            np.testing.assert_array_equal(lg, lcp_o[j, f])
            checked += 1
    assert checked > 0


@pytest.mark.parametrize("K", [8, 3])
def test_collisions_match_oracle(mom, K):
    wl = synth.tiny(22, n=2500, D=4, w=50, d=2, k=2, n_motifs=2)
    L = 5
    A, U = synth.hash_draws(wl.D, L, K, wl.w, 22)
    r = O.estimate_r(wl.series, wl.w, A)
    h, _, _ = make(mom, wl, L=L, K=K, r=r, hash_seed=22)
    keys_o, ok = agreeing_segments(h, wl, A, U, r, L)
    M = wl.n - wl.w + 1
    eps = wl.w // 2
    checked = 0
    for j in range(L):
        if not ok[j].all():
            continue
        for i in range(1, K + 1):
            allc = np.concatenate([O.colliding_pairs(keys_o[j, :, f], i) for f in range(wl.D)])
            u, W = np.unique(allc, return_counts=True)
            u = u[W >= wl.d]
            a, b = u // M, u % M
            ref = set(zip(a[(b - a) > eps].tolist(), b[(b - a) > eps].tolist()))
            got = h.collide(i, j)
            got_set = set(map(tuple, got.tolist()))
            assert len(got_set) == len(got)              # each pair once
            assert got_set == ref, (i, j)
            checked += 1
    assert checked > 0


# ---------------------------------------------------------- verification

@pytest.mark.parametrize("name", ["plain_small", "plain_fp32"])
def test_verify_matches_oracle(mom, name):
    wl = synth.plain_small(0) if name == "plain_small" else synth.plain_fp32(0, n=30_000)
    h, _, _ = make(mom, wl, L=2)
    M = wl.n - wl.w + 1
    rng = np.random.default_rng(0)
    pairs = rng.integers(0, M, size=(300, 2))
    pairs = np.concatenate([pairs, [[a, b] for a, b, _ in wl.planted if b < M]])
    per32, dd32, mask32 = h.verify(pairs, fp64=False)
    per64, dd64, mask64 = h.verify(pairs, fp64=True)
    for q, (a, b) in enumerate(pairs):
        ref = O.per_dim_distances(wl.series, wl.w, int(a), int(b))
        np.testing.assert_allclose(per64[q], ref, rtol=1e-9, atol=1e-9)
        np.testing.assert_allclose(per32[q], ref, rtol=1e-4, atol=1e-4)
        dd, dims, _ = O.select_d(ref, wl.d)
        assert dd64[q] == pytest.approx(dd, rel=1e-9, abs=1e-9)
        assert dd32[q] == pytest.approx(dd, rel=1e-4, abs=1e-4)
        srt = np.sort(ref)
        if wl.d < wl.D and srt[wl.d] - srt[wl.d - 1] > 1e-6 * max(1.0, srt[wl.d]):
            assert int(mask64[q]) == O.dims_mask(dims)


# ----------------------------------------------------------------- top-k

def assert_same_motifs(got, ref, rel=1e-9):
    assert [(m["a"], m["b"]) for m in got] == [(m[1], m[2]) for m in ref]
    for g, r in zip(got, ref):
        assert g["dist_d"] == pytest.approx(r[0], rel=rel, abs=1e-9)
        assert g["dims"] == tuple(r[3])
        assert g["dist_max"] == pytest.approx(r[4], rel=rel, abs=1e-9)


@pytest.mark.parametrize("seed,n,D,w,d,k", [(0, 300, 3, 20, 2, 3), (1, 700, 2, 33, 1, 2),
                                           (2, 1500, 4, 50, 2, 3), (3, 1031, 5, 64, 3, 2),
                                           (11, 900, 12, 40, 4, 2), (12, 700, 20, 30, 5, 2),
                                           (13, 500, 40, 24, 10, 2)])
def test_topk_exact_matches_oracle(mom, seed, n, D, w, d, k):
    wl = synth.tiny(seed, n=n, D=D, w=w, d=d, k=k, n_motifs=1)
    h, _, _ = make(mom, wl, L=2)
    got = h.topk_exact()
    ref = O.exact_topk(wl.series, wl.w, wl.d, wl.k)
    assert_same_motifs(got, ref)


@pytest.mark.parametrize("seed,n,D,w,d,k", [(21, 5000, 3, 64, 2, 3), (22, 4500, 8, 50, 3, 3),
                                           (23, 4200, 12, 40, 4, 2), (24, 3000, 20, 48, 5, 2),
                                           (25, 2600, 40, 32, 10, 2)])
def test_topk_exact_float32_matches_oracle(mom, seed, n, D, w, d, k):
    # float32 input takes the statistics sweeps: one lane per diagonal for
    # D <= 16 (padded to 4, 8, 16 dims), 16 dims per lane beyond (32, 64);
    # several row blocks of 2048 windows, diagonal blocks of 256 and a
    # ragged tail of both
    wl = synth.tiny(seed, n=n, D=D, w=w, d=d, k=k, n_motifs=2, dtype=np.float32)
    h, _, _ = make(mom, wl, L=2)
    got = h.topk_exact()
    ref = O.exact_topk(wl.series, wl.w, wl.d, wl.k)
    assert_same_motifs(got, ref)


@pytest.mark.parametrize("D,variant", [(3, 0), (3, 1), (3, 2), (8, 1), (8, 2), (12, 0), (12, 1),
                                       (12, 2), (20, 1), (40, 1)])
def test_sweep_variants_record_the_same_pairs(mom, D, variant, monkeypatch):
    # every form of the recording sweep the autotuner chooses from (the
    # statistics form with two stage heights, the slid form; for wide
    # series the statistics and slid wide forms) gives the exact top-k
    monkeypatch.setenv("MOMENTI_SWEEP_VARIANT", str(variant))
    wl = synth.tiny(30 + D, n=3500, D=D, w=48, d=max(1, D // 4), k=3, n_motifs=2, dtype=np.float32)
    h, _, _ = make(mom, wl, L=2)
    got = h.topk_exact()
    ref = O.exact_topk(wl.series, wl.w, wl.d, wl.k)
    assert_same_motifs(got, ref)


@pytest.mark.parametrize("D", [6, 24])
def test_topk_exact_float32_flat_windows(mom, D):
    # constant runs longer than a window: flat windows are the zero vector,
    # distance 0 to each other and sqrt(w) to any other window (so flat
    # pairs lead the top-k), and a run's level offset makes the neighbouring
    # windows' centring offsets large against their sigma; both take the
    # sweep's exact branch
    wl = synth.tiny(27, n=4000, D=D, w=40, d=2, k=4, n_motifs=1, dtype=np.float32)
    T = wl.series.copy()
    T[1, 1000:1150] = T[1, 1000]
    T[4, 2500:2600] = 7.5 + T[4, 2500]
    T[4, 3100:3180] = T[4, 3100]
    wl = synth.Workload(wl.name, np.ascontiguousarray(T), wl.w, wl.d, wl.k, wl.delta)
    h, _, _ = make(mom, wl, L=2)
    got = h.topk_exact()
    ref = O.exact_topk(wl.series, wl.w, wl.d, wl.k)
    assert_same_motifs(got, ref)


@pytest.mark.parametrize("seed", [1, 2, 4])
def test_topk_follows_algorithm_1(mom, seed):
    wl = synth.tiny(seed, 1500, 3, 50, 2, k=2, n_motifs=2)
    L = 100
    A, U = synth.hash_draws(wl.D, L, 8, wl.w, seed)
    r = O.estimate_r(wl.series, wl.w, A)
    # Algorithm 1's loop to its end (no cost switch)
    h, _, _ = make(mom, wl, L=L, r=r, hash_seed=seed, flags=mom.FLAG_NO_COST_SWITCH)
    got, st = h.topk()
    res = O.momenti(wl.series, wl.w, wl.d, wl.k, wl.delta, A, U, r)
    assert_same_motifs(got, res["motifs"])
    # The device keys equal the oracle's except for values in the float32
    # band around a bucket edge (about 0.2% of them here, checked by the
    # hash tests), which can move a collision by one repetition.  The
    # traversal itself is compared unconditionally: the oracle's Algorithm 1
    # loop run on the device's own keys must stop at the device's (i, j),
    # with the same TOP and the same Lemma stop bound.
    keys_dev = np.stack([h.keys(j) for j in range(L)])
    Z = [O.znorm_windows(wl.series[f], wl.w) for f in range(wl.D)]
    top, stop, _, _ = O.momenti_traverse(keys_dev, lambda a, b: O._pair_distances(Z, a, b),
                                         wl.d, wl.k, wl.delta, r, O.exclusion_zone(wl.w))
    assert (st["stop_i"], st["stop_j"]) == (stop or (0, 0))
    assert st["fallback"] == (stop is None)
    if stop is not None:
        assert_same_motifs(got, top)
        fb = O.failure_bound(top[-1][4], stop[0], stop[1], 8, L, wl.d, r)
        assert got[-1]["fail_bound"] == pytest.approx(fb, rel=1e-3)


def test_topk_plain_small_matches_exact(mom):
    path = os.path.join(GOLDEN, "exact_plain_small_seed0.json")
    gold = json.load(open(path))
    wl = synth.plain_small(0)
    h = mom.Momenti(w=wl.w, d=wl.d, k=wl.k, delta=wl.delta, precision=mom.PREC_FP32)
    h.hash_all(wl.series)
    got, st = h.topk()
    assert_same_motifs(got, gold["motifs"])
    assert st["L"] == 200 and st["K"] == 8
    ex = h.topk_exact()
    assert_same_motifs(ex, gold["motifs"])


@pytest.mark.parametrize("precision", ["fp32", "f16x2"])
def test_topk_plain_fp32_full_size_matches_exact(mom, precision):
    # the benchmark workload at full size (D=8, n=1e5, w=300, d=3, k=10):
    # the exact top-k written by tests/golden/make_golden.py (4.5 h of the
    # float64 oracle), with the library's default parameters
    gold = json.load(open(os.path.join(GOLDEN, "exact_plain_fp32_seed0.json")))
    wl = synth.plain_fp32(0)
    prec = mom.PREC_FP32 if precision == "fp32" else mom.PREC_F16X2
    h = mom.Momenti(w=wl.w, d=wl.d, k=wl.k, delta=wl.delta, mem_limit=wl.mem_limit,
                    precision=prec)
    h.hash_all(wl.series)
    got, st = h.topk()
    assert_same_motifs(got, gold["motifs"])
    assert st["max_rel_err_fp32"] < 1e-4
    h.close()


@pytest.mark.parametrize("seed,D,d", [(5, 4, 2), (6, 8, 3), (7, 6, 2)])
def test_subbucketed_and_tiled_collisions_agree(mom, seed, D, d):
    # prefix length 1 splits buckets by a second dimension; the tile form
    # checks every in-bucket pair: both must emit the same candidates
    wl = synth.tiny(seed, 2500, D, 40, d, k=4, n_motifs=1)
    L = 24
    A, U = synth.hash_draws(wl.D, L, 8, wl.w, seed)
    out = []
    for flags in (0, mom.FLAG_TILES_ONLY):
        h = mom.Momenti(w=wl.w, d=wl.d, k=wl.k, delta=wl.delta, K=8, L=L, r=0.0,
                        precision=mom.PREC_FP32, flags=flags | mom.FLAG_NO_COST_SWITCH)
        h.set_hash_params(A, U)
        h.hash_all(wl.series)
        motifs, st = h.topk()
        out.append((motifs, st))
    (m0, s0), (m1, s1) = out
    assert s0["n_candidates"] == s1["n_candidates"] > 0
    assert (s0["stop_i"], s0["stop_j"]) == (s1["stop_i"], s1["stop_j"])
    assert [(m["a"], m["b"]) for m in m0] == [(m["a"], m["b"]) for m in m1]
    ref = O.exact_topk(wl.series, wl.w, wl.d, wl.k)
    if s0["fallback"]:
        assert [(m["a"], m["b"]) for m in m0] == [(m[1], m[2]) for m in ref]


@pytest.mark.parametrize("seed,n,D,w,d,k", [(8, 2500, 3, 50, 1, 3), (9, 2000, 6, 40, 2, 4),
                                           (10, 1500, 12, 30, 4, 2)])
def test_cost_switch_keeps_the_exact_result(mom, seed, n, D, w, d, k):
    # the cost switch only moves the point where the exact path takes over;
    # with or without it the result is the exact top-k of the oracle (these
    # small, low-contrast cases never reach STOP)
    wl = synth.tiny(seed, n, D, w, d, k=k, n_motifs=1)
    ref = O.exact_topk(wl.series, wl.w, wl.d, wl.k)
    for flags in (0, mom.FLAG_NO_COST_SWITCH):
        h = mom.Momenti(w=wl.w, d=wl.d, k=wl.k, delta=wl.delta, precision=mom.PREC_FP32,
                        flags=flags)
        h.hash_all(wl.series)
        got, st = h.topk()
        if st["fallback"]:
            assert_same_motifs(got, ref)
        if flags:
            assert st["switch_level"] == 0
        elif st["switch_level"]:
            assert st["fallback"] == 1 and st["predicted_rest_ms"] > st["predicted_exact_ms"]
        h.close()
