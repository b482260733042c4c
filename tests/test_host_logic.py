"""Host arithmetic of the search, checked on the CPU against the oracle
(oracle/momenti_oracle.py): Eq. (eucl-collision-probability), the bound of
Lemma stop that Algorithm 2 compares with delta, and TOP of Algorithm 1 (the
greedy top-k under the trivial-match exclusion of Section 3.1) through the
pool the search keeps, fed in batches as verified pairs arrive.  These calls
use no device."""
import math

import numpy as np
import pytest

from oracle import momenti_oracle as O


@pytest.fixture(scope="module")
def mom():
    from paper_2502_14446_gb300 import build_ext
    build_ext.build()
    from paper_2502_14446_gb300 import momenti
    return momenti


def test_collision_probability_matches_the_oracle(mom):
    for R in (0.0, 1e-3, 0.5, 1.0, 2.5, 7.0, 30.0, 100.0):
        for r in (0.1, 0.6, 1.0, 4.0, 16.0):
            assert mom.collision_probability(R, r) == pytest.approx(
                O.collision_probability(R, r), rel=1e-12, abs=1e-15)


def test_failure_bound_matches_the_oracle(mom):
    for dist_max in (0.5, 2.0, 5.0):
        for i, K, L in ((8, 8, 200), (3, 8, 200), (1, 8, 200), (4, 4, 10)):
            for j in (0, 1, L // 2, L):
                for d in (1, 3):
                    for r in (0.6, 2.0):
                        got = mom.failure_bound(dist_max, i, j, K, L, d, r)
                        ref = O.failure_bound(dist_max, i, j, K, L, d, r)
                        assert got == pytest.approx(ref, rel=1e-12, abs=1e-300)


def test_failure_bound_rejects_out_of_range_indices(mom):
    assert math.isnan(mom.failure_bound(1.0, 0, 1, 8, 200, 1, 1.0))      # i < 1
    assert math.isnan(mom.failure_bound(1.0, 9, 1, 8, 200, 1, 1.0))      # i > K
    assert math.isnan(mom.failure_bound(1.0, 2, 201, 8, 200, 1, 1.0))    # j > L
    assert math.isnan(mom.failure_bound(1.0, 2, 1, 8, 200, 0, 1.0))      # d < 1
    assert math.isnan(mom.failure_bound(1.0, 2, 1, 8, 200, 1, 0.0))      # r <= 0
    assert math.isnan(mom.collision_probability(1.0, 0.0))
    assert math.isnan(mom.collision_probability(float("nan"), 1.0))
    assert mom.collision_probability(-1.0, 1.0) == 1.0


def _candidates(rng, m, M):
    """m distinct pairs a < b below M, with float32 distances on a coarse
    grid (many equal distances, so the (a, b) tie order matters)."""
    seen, a, b = set(), [], []
    while len(a) < m:
        x, y = sorted(int(v) for v in rng.integers(0, M, 2))
        if x < y and (x, y) not in seen:
            seen.add((x, y))
            a.append(x)
            b.append(y)
    dd = np.round(rng.uniform(0.0, 5.0, m), 1).astype(np.float32)
    return dd, np.array(a, np.int64), np.array(b, np.int64)


@pytest.mark.parametrize("seed", range(12))
def test_top_select_is_the_greedy_top_k(mom, seed):
    rng = np.random.default_rng(600 + seed)
    M = int(rng.integers(60, 3000))
    m = int(rng.integers(1, 500))
    dd, a, b = _candidates(rng, m, M)
    eps = int(rng.integers(0, 40))
    k = int(rng.integers(1, 15))
    ref = O.greedy_topk([(float(dd[q]), int(a[q]), int(b[q]), q) for q in range(m)], k, eps)
    for batch in (1, 7, int(rng.integers(1, m + 1)), m):
        assert mom.top_select(dd, a, b, k, eps, batch) == [c[3] for c in ref]


def test_top_select_keeps_first_occurrences(mom):
    # a pair verified again (same distance) is the same pair: TOP reports
    # its first position
    dd = np.array([3.0, 1.0, 2.0, 1.0, 0.5], np.float32)
    a = np.array([0, 100, 300, 100, 600], np.int64)
    b = np.array([50, 200, 400, 200, 700], np.int64)
    assert mom.top_select(dd, a, b, 3, 10, 2) == [4, 1, 2]


def test_top_select_argument_errors(mom):
    one = np.ones(1, np.float32)
    with pytest.raises(mom.MomentiError):
        mom.top_select(one, np.array([5]), np.array([5]), 1, 0)           # a >= b
    with pytest.raises(mom.MomentiError):
        mom.top_select(one, np.array([0]), np.array([5]), 1, -1)          # eps < 0
    with pytest.raises(mom.MomentiError):
        mom.top_select(np.array([np.nan], np.float32), np.array([0]), np.array([5]), 1, 0)
    with pytest.raises(mom.MomentiError):
        mom.top_select(one, np.array([0]), np.array([5]), 0, 0)           # k < 1
    assert mom.top_select(np.zeros(0, np.float32), np.zeros(0), np.zeros(0), 3, 0) == []


def test_top_select_through_pool_truncation(mom):
    # more candidates than the pool holds (2^22): it keeps the smaller half
    # and drops what lies above; TOP, far below that edge, is unchanged
    rng = np.random.default_rng(77)
    m, M = (1 << 22) + 300_000, 1 << 30
    a = rng.integers(0, M - 1000, m, dtype=np.int64)
    b = a + rng.integers(1, 1000, m, dtype=np.int64)
    key = a * M + b
    _, first = np.unique(key, return_index=True)
    first.sort()
    a, b = a[first], b[first]
    dd = rng.uniform(0.0, 100.0, a.size).astype(np.float32)
    k, eps = 10, 5
    order = np.lexsort((b, a, dd))[:20_000]          # (dd, a, b) order, a prefix
    ref = O.greedy_topk([(float(dd[q]), int(a[q]), int(b[q]), int(q)) for q in order], k, eps)
    assert len(ref) == k
    assert mom.top_select(dd, a, b, k, eps, 1 << 20) == [c[3] for c in ref]


def test_tensoring_bound_matches_the_oracle(mom):
    for p in (0.0, 0.3, 0.5, 0.8, 1.0):
        for K, L in ((8, 16), (8, 225), (4, 9), (2, 4)):
            for i in range(1, K + 1):
                for j in sorted({0, 1, L // 3, L // 2, L - 1, L}):
                    got = mom.tensoring_failure_bound(p, i, j, K, L)
                    ref = O.tensoring_failure_bound(p, i, j, K, L)
                    assert got == pytest.approx(ref, rel=1e-12, abs=1e-14), (p, i, j, K, L)
    for bad in ((0.5, 4, 1, 8, 200), (0.5, 0, 1, 8, 16), (0.5, 9, 1, 8, 16), (1.5, 4, 1, 8, 16),
                (0.5, 4, 17, 8, 16), (0.5, 3, 1, 7, 16), (0.5, 4, 0, 8, 0)):
        assert math.isnan(mom.tensoring_failure_bound(*bad)), bad
