"""Pins of the CPU oracle against the paper and the mathematics.

Each test checks the oracle against something other than itself: closed
forms of Eq. (zned), library statistics, brute force over subsets and pairs,
an independent integral form and a Monte Carlo simulation of Eq.
(eucl-collision-probability), hand-evaluated values of Algorithm 2, and the
control flow of the paper's Example 4.1.
"""
import itertools
import math

import numpy as np
import pytest

from oracle import momenti_oracle as O
from paper_2502_14446_gb300 import synth


# ---------------------------------------------------------------- Eq. (zned)

def test_zned_closed_forms():
    rng = np.random.default_rng(1)
    w = 57
    x = np.cumsum(rng.standard_normal(w))
    # shift/scale invariance: z-normalisation removes level and spread
    assert O.zned(x, 3.5 * x - 17.0) == pytest.approx(0.0, abs=1e-12)
    # a window and its negation are at the maximum distance 2 sqrt(w)
    assert O.zned(x, -x) == pytest.approx(2.0 * math.sqrt(w), rel=1e-12)
    y = np.cumsum(rng.standard_normal(w))
    dxy = O.zned(x, y)
    assert dxy == pytest.approx(O.zned(y, x), rel=1e-14)
    assert 0.0 <= dxy <= 2.0 * math.sqrt(w) + 1e-12


def test_zned_pearson_identity():
    # Section 2: dist^2 = 2 w (1 - corr) with the population sigma;
    # corr from numpy's corrcoef (independent code)
    rng = np.random.default_rng(2)
    for w in (8, 100, 301):
        x = rng.standard_normal(w).cumsum()
        y = rng.standard_normal(w).cumsum() + 0.3 * x
        corr = np.corrcoef(x, y)[0, 1]
        assert O.zned(x, y) ** 2 == pytest.approx(2 * w * (1 - corr), rel=1e-10)


def test_zned_flat_windows():
    w = 20
    flat = np.full(w, 4.25)
    x = np.arange(w, dtype=float) ** 1.5
    assert O.zned(flat, flat + 3.0) == 0.0
    assert O.zned(flat, x) == pytest.approx(math.sqrt(w), rel=1e-12)


def test_window_stats_against_numpy():
    rng = np.random.default_rng(3)
    x = rng.standard_normal(500).cumsum() * 10 + 1e3
    w = 37
    mu, sd, flat = O.window_stats(x, w)
    for a in (0, 1, 100, 463):
        assert mu[a] == pytest.approx(np.mean(x[a:a + w]), rel=1e-13)
        assert sd[a] == pytest.approx(np.std(x[a:a + w]), rel=1e-11)
    assert not flat.any()
    x[200:260] = 7.0
    _, _, flat = O.window_stats(x, w)
    assert flat[200:224].all() and not flat[199] and not flat[224]


def test_znorm_windows_rows():
    rng = np.random.default_rng(4)
    x = rng.standard_normal(300).cumsum()
    Z = O.znorm_windows(x, 50)
    assert Z.shape == (251, 50)
    assert np.allclose(Z.mean(axis=1), 0, atol=1e-12)
    assert np.allclose((Z * Z).sum(axis=1), 50, rtol=1e-12)
    assert O.zned(x[10:60], x[70:120]) == pytest.approx(np.linalg.norm(Z[10] - Z[70]), rel=1e-12)


# ----------------------------------------------- Definition distdims, dims_d

def test_select_d_against_subset_minimum():
    rng = np.random.default_rng(5)
    for trial in range(200):
        D = int(rng.integers(1, 7))
        d = int(rng.integers(1, D + 1))
        dist = rng.random(D) * 5
        if trial % 3 == 0:
            dist = np.round(dist)          # ties
        best = min(itertools.combinations(range(D), d),
                   key=lambda F: (sum(dist[f] for f in F), F))
        dd, dims, dmax = O.select_d(dist, d)
        assert dd == pytest.approx(sum(dist[f] for f in best), abs=1e-12)
        assert dmax == pytest.approx(max(dist[f] for f in dims), abs=0)
        if len(set(np.round(dist, 12))) == D:
            assert dims == best


# ------------------------------------------------------- top-k definitions

@pytest.mark.parametrize("seed", [0, 1, 2])
def test_exact_topk_equals_naive_enumeration(seed):
    wl = synth.tiny(seed, n=150, D=3, w=12, d=2, k=3, n_motifs=1)
    naive = O.naive_topk(wl.series, wl.w, wl.d, wl.k)
    ex = O.exact_topk(wl.series, wl.w, wl.d, wl.k, block=37)
    assert [(m[1], m[2]) for m in naive] == [(m[1], m[2]) for m in ex]
    for a, b in zip(naive, ex):
        assert a[0] == pytest.approx(b[0], rel=1e-9)
        assert a[3] == b[3]
        assert a[4] == pytest.approx(b[4], rel=1e-9)


def test_exact_topk_threshold_and_invariants():
    wl = synth.tiny(7, n=900, D=4, w=40, d=2, k=4, n_motifs=2)
    full = O.exact_topk(wl.series, wl.w, wl.d, wl.k)
    thr = O.exact_topk_auto(wl.series, wl.w, wl.d, wl.k, tau0=0.5)
    assert [(m[1], m[2]) for m in full] == [(m[1], m[2]) for m in thr]
    eps = wl.w // 2
    ends = [x for m in full for x in (m[1], m[2])]
    for i in range(len(ends)):
        for j in range(i + 1, len(ends)):
            assert abs(ends[i] - ends[j]) > eps          # no trivial matches
    dd = [m[0] for m in full]
    assert dd == sorted(dd)
    for m in full:                                       # recomputed one by one
        dist = O.per_dim_distances(wl.series, wl.w, m[1], m[2])
        assert O.select_d(dist, wl.d)[0] == pytest.approx(m[0], rel=1e-10)
    # the planted pairs are the two best motifs
    assert {(m[1], m[2]) for m in full[:2]} == {(a, b) for a, b, _ in wl.planted}


def test_greedy_exclusion_non_monotone():
    # one close pair displaces two accepted ones: the k-th distance grows
    eps = 5
    base = [(1.0, 0, 100, None), (2.0, 50, 200, None), (3.0, 300, 400, None)]
    top = O.greedy_topk(base, 2, eps)
    assert [(c[1], c[2]) for c in top] == [(0, 100), (50, 200)]
    top = O.greedy_topk(base + [(0.5, 2, 52, None)], 2, eps)
    assert [(c[1], c[2]) for c in top] == [(2, 52), (300, 400)]


# ------------------------------------- Eq. (eucl-collision-probability)

def _collision_integral(R, r):
    # Datar et al.'s integral form: int_0^r (1/R) f(t/R) (1 - t/r) dt with f
    # the density of |N(0,1)|
    from scipy.integrate import quad
    f = lambda t: 2.0 / math.sqrt(2 * math.pi) * math.exp(-(t / R) ** 2 / 2) / R * (1 - t / r)
    return quad(f, 0.0, r)[0]


@pytest.mark.parametrize("ratio", [0.05, 0.3, 1.0, 2.0, 7.0])
def test_collision_probability_integral_form(ratio):
    r = 1.7
    R = r / ratio
    assert O.collision_probability(R, r) == pytest.approx(_collision_integral(R, r), rel=1e-9)


def test_collision_probability_monte_carlo():
    rng = np.random.default_rng(11)
    w, S, r = 32, 200_000, 1.0
    for ratio in (0.5, 1.0, 2.0, 4.0):
        R = r / ratio
        x = rng.standard_normal(w)
        u = rng.standard_normal(w)
        y = x + R * u / np.linalg.norm(u)
        a = rng.standard_normal((S, w))
        b = rng.random(S) * r
        hit = np.floor((a @ x + b) / r) == np.floor((a @ y + b) / r)
        p = O.collision_probability(R, r)
        assert abs(hit.mean() - p) < 4 * math.sqrt(p * (1 - p) / S)


def test_collision_probability_limits():
    assert O.collision_probability(0.0, 1.0) == 1.0
    assert O.collision_probability(1e9, 1.0) < 1e-8
    vals = [O.collision_probability(R, 0.8) for R in np.linspace(0.01, 20, 300)]
    assert all(x > y for x, y in zip(vals, vals[1:]))


# ------------------------------------------------------------ Algorithm 2

def _R_for(P, r):
    lo, hi = 1e-6, 1e6
    for _ in range(200):
        mid = math.sqrt(lo * hi)
        if O.collision_probability(mid, r) > P:
            lo = mid
        else:
            hi = mid
    return lo


def test_stop_hand_evaluated():
    r, K, L, d = 1.0, 8, 10, 2
    R = _R_for(0.5, r)                  # P(R) = 0.5, so p = 0.25 at d = 2
    p = 0.25
    assert O.failure_bound(R, K, 3, K, L, d, r) == pytest.approx((1 - p ** 8) ** 3, rel=1e-8)
    assert O.failure_bound(R, 2, 4, K, L, d, r) == pytest.approx(
        (1 - p ** 2) ** 4 * (1 - p ** 3) ** 6, rel=1e-8)
    # (15/16)^j (63/64)^(10 - j): 0.5507 at j = 9, 0.5245 at j = 10
    assert not O.stop_condition(R, 2, 9, K, L, d, 0.53, r)
    assert O.stop_condition(R, 2, 10, K, L, d, 0.53, r)
    # distance 0 (p = 1) stops at once; a far pair never stops
    assert O.stop_condition(0.0, K, 1, K, L, d, 1e-9, r)
    assert not O.stop_condition(1e9, 1, L, K, L, d, 0.5, r)


def test_example_4_1_control_flow():
    """Example 4.1: K=4, L=2, delta=0.1, k=1; only the two motif pairs ever
    collide, in d=2 dimensions; TOP fails STOP at every iteration of i=4,
    re-evaluates both pairs at i=3 and stops at (i, j) = (3, 2)."""
    K, L, D, d, M, delta = 4, 2, 3, 2, 40, 0.1
    # p = P(dist^max)^2 in (0.8835, 0.8897) makes (3, 2) the first stop
    r = 1.0
    Rmax = _R_for(math.sqrt(0.886), r)
    keys = np.zeros((L, M, D), dtype=np.uint64)
    for j in range(L):
        for f in range(D):
            for a in range(M):
                keys[j, a, f] = np.uint64(((a * 7 + f * 3 + j) % 256) << 56 | (a << 8))
    ab, cd = (3, 30), (8, 25)
    for j in range(L):
        for f in (0, 2):
            for x, y in (ab, cd):
                keys[j, y, f] = keys[j, x, f]
    dist = {ab: [0.5 * Rmax, 9.0, Rmax], cd: [Rmax, 9.0, 1.2 * Rmax]}
    calls = []

    def pair_dist(a, b):
        calls.append(len(a))
        return np.array([dist[(int(x), int(y))] for x, y in zip(a, b)]).T

    top, stop, n_dist, pool = O.momenti_traverse(keys, pair_dist, d, 1, delta, r, eps=2, K=K)
    assert stop == (3, 2)
    assert [(m[1], m[2]) for m in top] == [ab]
    assert n_dist == 8 and calls == [2, 2, 2, 2]
    assert pool == 2


# --------------------------------------------------- Eq. (drp) and the index

def test_hash_values_direct():
    wl = synth.tiny(3, n=400, D=2, w=30, d=1, n_motifs=0)
    A, U = synth.hash_draws(2, 3, 4, 30, 3)
    r = 0.37
    h, t = O.hash_values(wl.series, 30, A, U, r, 1)
    for a in (0, 17, 370):
        x = wl.series[1, a:a + 30]
        z = (x - x.mean()) / x.std()
        for j in range(3):
            for kk in range(4):
                val = (A[1, j, kk].astype(np.float64) @ z + float(U[1, j, kk]) * r) / r
                assert t[a, j, kk] == pytest.approx(val, rel=1e-12, abs=1e-12)
                assert h[a, j, kk] == max(-128, min(127, math.floor(val)))


def test_pack_keys_is_lexicographic():
    rng = np.random.default_rng(8)
    for K in (1, 3, 8):
        h = rng.integers(-128, 128, size=(500, K))
        h[::7, 0] = 0
        keys = O.pack_keys(h)
        by_key = sorted(range(500), key=lambda q: (int(keys[q]), q))
        by_tuple = sorted(range(500), key=lambda q: (tuple(h[q]), q))
        assert by_key == by_tuple
        for i in range(1, K + 1):
            pre = O.prefix(keys, i)
            for q in range(0, 500, 37):
                same = [s for s in range(500) if tuple(h[s, :i]) == tuple(h[q, :i])]
                assert sorted(np.nonzero(pre == pre[q])[0].tolist()) == same
        if K < 8:
            assert (keys & np.uint64((1 << (64 - 8 * K)) - 1) == 0).all()


def test_build_index_against_sorted_tuples():
    rng = np.random.default_rng(9)
    L, M, D = 2, 300, 2
    h = rng.integers(-3, 3, size=(L, M, D, 8))        # many ties and shared prefixes
    keys = O.pack_keys(h)
    order, lcp = O.build_index(keys)
    for j in range(L):
        for f in range(D):
            ref = sorted(range(M), key=lambda a: (tuple(h[j, a, f]), a))
            assert order[j, f].tolist() == ref
            for p in range(1, M):
                u, v = h[j, ref[p - 1], f], h[j, ref[p], f]
                n_eq = 0
                while n_eq < 8 and u[n_eq] == v[n_eq]:
                    n_eq += 1
                assert lcp[j, f, p] == n_eq


def test_colliding_pairs_brute_force():
    rng = np.random.default_rng(10)
    M = 120
    h = rng.integers(-2, 2, size=(M, 8))
    keys = O.pack_keys(h)
    for i in (1, 2, 3):
        got = set(O.colliding_pairs(keys, i).tolist())
        ref = {a * M + b for a in range(M) for b in range(a + 1, M)
               if tuple(h[a, :i]) == tuple(h[b, :i])}
        assert got == ref


# ------------------------------------------------------ Section 6.1: r

def test_estimate_r_bounds_and_invariance():
    wl = synth.tiny(4, n=3000, D=3, w=64, d=2, n_motifs=0)
    A, U = synth.hash_draws(3, 2, 8, 64, 4)
    r = O.estimate_r(wl.series, 64, A)
    # |a . z| <= |a| |z| = |a| sqrt(w) (Cauchy-Schwarz, |z|^2 = w)
    amax = max(np.linalg.norm(A[f, 0, kk]) for f in range(3) for kk in range(8))
    assert 0 < r <= 2 * amax * math.sqrt(64) / 256
    # z-normalised projections of a random-walk sample spread over several
    # sigma = sqrt(w): the 256 buckets cover at least +-3 sqrt(w)
    assert r * 256 > 6 * math.sqrt(64)
    r2 = O.estimate_r(5.0 * wl.series - 40.0, 64, A)
    assert r2 == pytest.approx(r, rel=1e-10)


def test_estimate_r_hand_computed():
    # w = 2: a rising window z-normalises to (-1, 1), a falling one to
    # (1, -1) (population sigma = half the step), so each projection is
    # +-(a_1 - a_0) and the heuristic of Section 6.1 can be written out by
    # hand.  Dim 0 rises twice: projections a_1 - a_0 = 3 and 1 for the two
    # vectors of repetition 0.  Dim 1 falls then rises: 2, 0, then -2, 0.
    # Pooled over both dims the range is 3 - (-2) = 5, so r = 5 / 256.
    # Per-dim ranges are 2 and 4 (largest 4, mean 3); dividing by 255 gives
    # 5 / 255: each of those misreadings fails the equality below.
    T = np.array([[0.0, 1.0, 3.0],
                  [5.0, 2.0, 4.0]])
    A = np.zeros((2, 2, 2, 2))
    A[0, 0] = [[0.0, 3.0], [0.0, 1.0]]
    A[1, 0] = [[2.0, 0.0], [1.0, 1.0]]
    A[:, 1] = 100.0                    # repetition 1 is not part of the sample
    assert O.estimate_r(T, 2, A) == pytest.approx(5.0 / 256.0, rel=1e-12)


def test_estimate_r_uses_the_evenly_spaced_sample():
    # M = 5 windows, a sample of 3: positions floor(q (M - 1) / 2) = 0, 2, 4.
    # Those windows rise (projection a_1 - a_0 = 2 for the one vector that
    # is not constant zero, 0 for the other); window 1, left out of the
    # sample, falls (projection -2).  With the sample the range is
    # 2 - 0 = 2 (r = 2/256); a sample that took window 1 would give 4/256.
    T = np.array([[0.0, 1.0, 0.5, 2.0, 3.0, 4.0]])
    A = np.zeros((1, 1, 2, 2))
    A[0, 0, 0] = [0.0, 2.0]
    assert list(O.sample_positions(5, 3)) == [0, 2, 4]
    assert O.estimate_r(T, 2, A, samples=3) == pytest.approx(2.0 / 256.0, rel=1e-12)
    assert O.estimate_r(T, 2, A, samples=5) == pytest.approx(4.0 / 256.0, rel=1e-12)


# ----------------------------------------------------------- Algorithm 1

@pytest.mark.parametrize("seed", [1, 2])
def test_momenti_matches_exact_on_small_series(seed):
    wl = synth.tiny(seed, 1500, 3, 50, 2, k=2, n_motifs=2)
    A, U = synth.hash_draws(wl.D, 100, 8, wl.w, seed)
    r = O.estimate_r(wl.series, wl.w, A)
    res = O.momenti(wl.series, wl.w, wl.d, wl.k, wl.delta, A, U, r)
    ex = O.exact_topk(wl.series, wl.w, wl.d, wl.k)
    assert res["stop"] is not None
    assert res["fail_bound"] <= wl.delta
    assert [(m[1], m[2]) for m in res["motifs"]] == [(m[1], m[2]) for m in ex]
    assert {(m[1], m[2]) for m in ex} == {(a, b) for a, b, _ in wl.planted}


# --------------------------------------- Section 6.3: several dimensionalities

def test_multi_with_one_dimensionality_is_algorithm_1():
    wl = synth.tiny(1, 1500, 3, 50, 2, k=2, n_motifs=2)
    A, U = synth.hash_draws(wl.D, 100, 8, wl.w, 1)
    r = O.estimate_r(wl.series, wl.w, A)
    one = O.momenti(wl.series, wl.w, 2, wl.k, wl.delta, A, U, r)
    multi = O.momenti_multi(wl.series, wl.w, 2, 2, wl.k, wl.delta, A, U, r)
    assert one["stop"] is not None
    assert multi[2]["stop"] == one["stop"] and multi[2]["motifs"] == one["motifs"]
    assert multi[2]["fail_bound"] == one["fail_bound"] and multi["n_dist"] == one["n_dist"]


def test_multi_when_every_pair_collides_at_once():
    # r far above every projection and offsets b = r / 2: every hash value
    # is floor(1/2 + tiny) = 0, every pair collides in every dim at (K, 1),
    # each TOP is the exact top-k at once and STOP holds for every d there
    wl = synth.tiny(9, 400, 3, 30, 1, k=2, n_motifs=0)
    A, U = synth.hash_draws(wl.D, 4, 8, wl.w, 9)
    U = np.full_like(U, 0.5)
    multi = O.momenti_multi(wl.series, wl.w, 1, 3, wl.k, 0.1, A, U, 1e9)
    for d in (1, 2, 3):
        assert multi[d]["stop"] == (8, 1)
        ref = O.naive_topk(wl.series, wl.w, d, wl.k)
        assert [(m[1], m[2], tuple(m[3])) for m in multi[d]["motifs"]] == \
               [(m[1], m[2], tuple(m[3])) for m in ref]


def test_multi_without_stop_is_exact_and_collides_at_the_lowest_d():
    # delta too small for STOP: every d ends in the exact top-k, and the
    # collision threshold stays at d_low (as many distance computations as
    # the single search for d_low)
    wl = synth.tiny(10, 400, 3, 30, 1, k=2, n_motifs=1)
    A, U = synth.hash_draws(wl.D, 3, 8, wl.w, 10)
    r = O.estimate_r(wl.series, wl.w, A)
    multi = O.momenti_multi(wl.series, wl.w, 1, 3, wl.k, 1e-300, A, U, r)
    one = O.momenti(wl.series, wl.w, 1, wl.k, 1e-300, A, U, r)
    assert one["stop"] is None and multi["n_dist"] == one["n_dist"]
    for d in (1, 2, 3):
        assert multi[d]["stop"] is None and multi[d]["fail_bound"] == 0.0
        ref = O.naive_topk(wl.series, wl.w, d, wl.k)
        assert [(m[1], m[2], tuple(m[3])) for m in multi[d]["motifs"]] == \
               [(m[1], m[2], tuple(m[3])) for m in ref]


def test_multi_confirms_each_dimensionality_by_its_own_bound():
    wl = synth.tiny(2, 1500, 3, 50, 2, k=2, n_motifs=2)
    A, U = synth.hash_draws(wl.D, 100, 8, wl.w, 2)
    r = O.estimate_r(wl.series, wl.w, A)
    multi = O.momenti_multi(wl.series, wl.w, 1, 3, wl.k, wl.delta, A, U, r)
    confirmed = [d for d in (1, 2, 3) if multi[d]["stop"] is not None]
    assert confirmed
    for d in confirmed:
        i, j = multi[d]["stop"]
        top = multi[d]["motifs"]
        assert len(top) == wl.k
        fb = O.failure_bound(top[-1][4], i, j, 8, 100, d, r)
        assert multi[d]["fail_bound"] == fb and fb <= wl.delta


# ------------------------------------------- Section 6.1: tensoring bound

def _tensoring_miss_mc(p, i, j, K, L, trials, rng):
    """Direct simulation of the tensored hash collisions of one pair: each
    of the m left and m right functions has K/2 values, each colliding
    with probability p; repetition j' (0-based) pairs left j' div m with
    right j' mod m and interleaves them (left first); prefix length t
    collides iff its first t interleaved values all collide.  Counts the
    trials in which none of the first j repetitions collides at length i
    and (for i < K) none of the L repetitions collides at length i + 1."""
    m = math.isqrt(L)
    half = K // 2
    left = rng.random((trials, m, half)) < p
    right = rng.random((trials, m, half)) < p
    inter = np.empty((trials, m, m, K), bool)
    inter[..., 0::2] = left[:, :, None, :]
    inter[..., 1::2] = right[:, None, :, :]
    pref = np.cumprod(inter, axis=-1).astype(bool)          # pref[..., t-1]: length t collides
    rep = np.arange(L)
    hit_i = pref[:, rep // m, rep % m, i - 1][:, :j].any(axis=1)
    hit = hit_i
    if i < K:
        hit = hit | pref[:, rep // m, rep % m, i].any(axis=1)
    return 1.0 - hit.mean()


@pytest.mark.parametrize("p,i,j,K,L", [
    (0.5, 4, 5, 8, 16), (0.5, 3, 9, 8, 16), (0.7, 8, 7, 8, 16), (0.6, 1, 2, 8, 9),
    (0.8, 6, 0, 8, 9), (0.4, 2, 16, 8, 16), (0.9, 7, 20, 8, 25), (0.5, 8, 16, 8, 16)])
def test_tensoring_bound_is_the_simulated_miss_probability(p, i, j, K, L):
    rng = np.random.default_rng(hash((p, i, j, K, L)) % 2**32)
    trials = 200_000
    mc = _tensoring_miss_mc(p, i, j, K, L, trials, rng)
    exact = O.tensoring_failure_bound(p, i, j, K, L)
    sigma = math.sqrt(max(exact * (1 - exact), 1e-12) / trials)
    assert abs(mc - exact) <= 5 * sigma + 1e-9


def test_tensoring_bound_special_cases():
    # nothing visited: certain miss; p = 1: any visit collides
    assert O.tensoring_failure_bound(0.5, 8, 0, 8, 16) == pytest.approx(1.0)
    assert O.tensoring_failure_bound(1.0, 5, 3, 8, 16) == pytest.approx(0.0, abs=1e-15)
    # one repetition at the top level: the interleaved K values all collide
    assert O.tensoring_failure_bound(0.6, 8, 1, 8, 16) == pytest.approx(1 - 0.6 ** 8)
    # more repetitions and a larger p never raise the miss probability
    seq = [O.tensoring_failure_bound(0.5, 4, j, 8, 16) for j in range(17)]
    assert all(x >= y - 1e-15 for x, y in zip(seq, seq[1:]))
    ps = [O.tensoring_failure_bound(p, 4, 6, 8, 16) for p in (0.3, 0.5, 0.7, 0.9)]
    assert all(x >= y for x, y in zip(ps, ps[1:]))
    with pytest.raises(ValueError):
        O.tensoring_failure_bound(0.5, 4, 1, 8, 200)          # L not a square
    with pytest.raises(ValueError):
        O.tensoring_failure_bound(0.5, 4, 0, 8, 0)            # no repetitions


def test_printed_tensoring_lemma_is_not_a_bound():
    # the lemma's P_t(i/2, j) = (1 - p^ceil(i/2))^(j div m) (1 - p^floor(i/2))^(j mod m)
    # at i = K falls below the simulated and re-derived miss probability
    p, K, L, m = 0.5, 8, 16, 4
    for j in (4, 8, 12):
        printed = (1 - p ** 4) ** (j // m) * (1 - p ** 4) ** (j % m)
        assert O.tensoring_failure_bound(p, K, j, K, L) > printed + 0.04


def _tensored_draws(D, m, K, w, seed):
    Al, Ul = synth.hash_draws(D, m, K // 2, w, seed)
    Ar, Ur = synth.hash_draws(D, m, K // 2, w, seed + 1000)
    return Al, Ul, Ar, Ur


def test_tensored_keys_are_keys_of_interleaved_functions():
    # repetition j' = (l, r) is the plain composite hash of the functions
    # whose values alternate left l and right r
    wl = synth.tiny(12, 600, 2, 40, 1, n_motifs=0)
    m, K = 3, 8
    Al, Ul, Ar, Ur = _tensored_draws(wl.D, m, K, wl.w, 12)
    r = O.estimate_r(wl.series, wl.w, Al)
    A = np.empty((wl.D, m * m, K, wl.w), np.float32)
    U = np.empty((wl.D, m * m, K), np.float32)
    for jj in range(m * m):
        lf, rf = divmod(jj, m)
        A[:, jj, 0::2], A[:, jj, 1::2] = Al[:, lf], Ar[:, rf]
        U[:, jj, 0::2], U[:, jj, 1::2] = Ul[:, lf], Ur[:, rf]
    plain, t = O.hash_all(wl.series, wl.w, A, U, r)
    tens = O.tensored_keys(wl.series, wl.w, Al, Ul, Ar, Ur, r)
    # equal except where a value sits within rounding of a bucket edge
    near = (np.abs(t - np.round(t)) < 1e-9).any(axis=-1).transpose(2, 1, 0)   # (L, M, D)
    assert np.array_equal(tens[~near], plain[~near]) and near.mean() < 1e-3


def test_tensored_search_stops_on_its_bound_or_is_exact():
    # close planted motifs (noise 0.01), m = 15 (L = 225), delta = 0.2:
    # STOP holds on these seeds; the result is the exact top-k either way
    stopped = 0
    for seed in (1, 2, 3):
        wl = synth.tiny(seed, 1500, 3, 50, 2, k=2, n_motifs=2, noise=0.01)
        Al, Ul, Ar, Ur = _tensored_draws(wl.D, 15, 8, wl.w, seed)
        r = O.estimate_r(wl.series, wl.w, Al)
        res = O.momenti_tensored(wl.series, wl.w, wl.d, wl.k, 0.2, Al, Ul, Ar, Ur, r)
        ex = O.exact_topk(wl.series, wl.w, wl.d, wl.k)
        assert [(m[1], m[2]) for m in res["motifs"]] == [(m[1], m[2]) for m in ex]
        if res["stop"] is not None:
            stopped += 1
            i, j = res["stop"]
            p = O.collision_probability(res["motifs"][-1][4], r) ** wl.d
            assert res["fail_bound"] == O.tensoring_failure_bound(p, i, j, 8, 225) <= 0.2
    assert stopped >= 2


# ------------------------- the oracle's C pair enumeration (exact_pairs.c)

def _same_topk(got, ref, rel=1e-9):
    assert [(g[1], g[2], tuple(g[3])) for g in got] == [(r[1], r[2], tuple(r[3])) for r in ref]
    for g, r in zip(got, ref):
        assert g[0] == pytest.approx(r[0], rel=rel, abs=1e-9)
        assert g[4] == pytest.approx(r[4], rel=rel, abs=1e-9)


@pytest.mark.parametrize("seed,n,D,w,d,k", [(0, 300, 3, 20, 2, 3), (1, 700, 2, 33, 1, 2),
                                           (2, 1500, 4, 50, 2, 3), (11, 900, 12, 40, 4, 2),
                                           (13, 500, 40, 24, 10, 2), (14, 400, 5, 30, 5, 3)])
def test_diagonal_enumeration_matches_the_matrix_form(seed, n, D, w, d, k):
    # exact_topk forms every dot product with a matrix product; the C code
    # slides them along diagonals: the same top-k (pairs, dims, distances)
    wl = synth.tiny(seed, n=n, D=D, w=w, d=d, k=k, n_motifs=1)
    _same_topk(O.exact_topk_diag(wl.series, w, d, k), O.exact_topk(wl.series, w, d, k))


def test_diagonal_enumeration_matches_the_definitions_on_tiny_series():
    for seed in (3, 4):
        wl = synth.tiny(seed, n=90, D=3, w=12, d=2, k=2, n_motifs=1)
        _same_topk(O.exact_topk_diag(wl.series, wl.w, 2, 2), O.naive_topk(wl.series, wl.w, 2, 2))


def test_diagonal_recurrence_over_long_diagonals():
    # n - w >> 1024: the slid dot products are recomputed every 1024 steps
    # and must still agree with the direct ones (float64)
    wl = synth.tiny(15, n=6000, D=2, w=16, d=1, k=3, n_motifs=1)
    wl.series[:, :] += 1e3          # a large level stresses the Pearson form's cancellation
    _same_topk(O.exact_topk_diag(wl.series, wl.w, 1, 3), O.exact_topk(wl.series, wl.w, 1, 3),
               rel=1e-7)


def test_pairs_below_is_every_pair_below_the_threshold():
    wl = synth.tiny(5, n=120, D=3, w=10, d=2, k=1, n_motifs=0)
    tau = 5.0
    got = O.pairs_below(wl.series, wl.w, 2, tau)
    ref = []
    M, eps = wl.n - wl.w + 1, O.exclusion_zone(wl.w)
    for a in range(M):
        for b in range(a + eps + 1, M):
            dd, dims, mx = O.select_d(O.per_dim_distances(wl.series, wl.w, a, b), 2)
            if dd <= tau:
                ref.append((a, b, dd, O.dims_mask(dims), mx))
    assert len(got) == len(ref) > 10
    ref.sort(key=lambda x: (x[2], x[0], x[1]))
    for g, r in zip(got, ref):
        assert (int(g["a"]), int(g["b"]), int(g["dims"])) == (r[0], r[1], r[3])
        assert g["dist_d"] == pytest.approx(r[2], rel=1e-9)
        assert g["dist_max"] == pytest.approx(r[4], rel=1e-9)


def test_diagonal_enumeration_of_flat_windows():
    # flat windows z-normalise to zero: distance 0 between two of them,
    # sqrt(w) to any other (reading 2), as in znorm_windows
    rng = np.random.default_rng(3)
    T = np.cumsum(rng.standard_normal((2, 400)), axis=1)
    T[0, 50:120] = 7.0
    T[0, 250:330] = -2.0
    got = O.exact_topk_diag(T, 20, 1, 3)
    _same_topk(got, O.exact_topk(T, 20, 1, 3))
    assert got[0][0] == 0.0
