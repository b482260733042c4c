"""The seeded input generators (paper_2502_14446_gb300/synth.py) on the
CPU: each workload has the stated shape, parameters and element type, the
same seed gives the same numbers, planted motifs sit where the recipe puts
them and are close pairs in their dims, and the hash draws have the stated
ranges (projection entries half-representable, offsets in [0, 1))."""
import math

import numpy as np
import pytest

from oracle import momenti_oracle as O
from paper_2502_14446_gb300 import synth


def test_pick_offsets_spacing_and_range():
    rng = synth._rng(11)
    for count, n, w, gap in ((2, 5000, 100, 200), (10, 3000, 50, 100), (6, 1300, 50, 200)):
        offs = synth._pick_offsets(rng, count, n, w, gap)
        assert len(offs) == count
        assert all(0 <= o <= n - w for o in offs)
        assert all(offs[i + 1] - offs[i] >= gap for i in range(count - 1))
    with pytest.raises(ValueError):
        synth._pick_offsets(rng, 10, 500, 50, 100)        # no room for the gaps


def test_planted_motifs_are_close_pairs():
    wl = synth.tiny(21, 4000, 4, 60, 2, k=3, n_motifs=3)
    assert len(wl.planted) == 3
    starts = sorted(x for a, b, _ in wl.planted for x in (a, b))
    assert all(starts[i + 1] - starts[i] >= 2 * wl.w for i in range(len(starts) - 1))
    rng = np.random.default_rng(5)
    M = wl.n - wl.w + 1
    for a, b, dims in wl.planted:
        assert a < b and len(dims) == wl.d and len(set(dims)) == wl.d
        planted = O.per_dim_distances(wl.series, wl.w, a, b)[list(dims)]
        # random pairs of windows in the same dims, for scale
        other = [O.per_dim_distances(wl.series, wl.w, int(x), int(y))[list(dims)].mean()
                 for x, y in rng.integers(0, M, (50, 2)) if abs(int(x) - int(y)) > wl.w]
        assert planted.max() < 0.25 * np.median(other)


def test_same_seed_same_numbers():
    a, b = synth.tiny(3, 900, 3, 40, 2), synth.tiny(3, 900, 3, 40, 2)
    assert np.array_equal(a.series, b.series) and a.planted == b.planted
    c = synth.tiny(4, 900, 3, 40, 2)
    assert not np.array_equal(a.series, c.series)


def test_plain_fp32_recipe():
    wl = synth.plain_fp32(0)
    assert wl.series.shape == (8, 100_000) and wl.series.dtype == np.float32
    assert wl.series.flags.c_contiguous
    assert (wl.w, wl.d, wl.k, wl.delta, wl.mem_limit) == (300, 3, 10, 0.05, 8 << 30)
    assert len(wl.planted) == 5 and all(len(dims) == 3 for _, _, dims in wl.planted)


def test_batch_form_recipe():
    wls = synth.batch_form(0, count=24)
    assert len(wls) == 24
    for wl in wls:
        assert wl.series.dtype == np.float32 and wl.series.flags.c_contiguous
        assert 3 <= wl.D <= 16 and wl.w in (50, 100, 200)
        assert wl.d == math.ceil(wl.D / 3) and (wl.k, wl.delta) == (5, 0.05)
        assert 2000 <= wl.n <= 200_000 or wl.n == 8 * wl.w + 16
        assert len(wl.planted) == 2
    # log-uniform lengths: both ends of the range are drawn
    ns = [wl.n for wl in wls]
    assert min(ns) < 20_000 and max(ns) > 20_000


def test_hash_draws_ranges():
    A, U = synth.hash_draws(3, 4, 8, 50, seed=2)
    assert A.shape == (3, 4, 8, 50) and U.shape == (3, 4, 8)
    assert A.dtype == np.float32 and U.dtype == np.float32
    assert np.array_equal(A, A.astype(np.float16).astype(np.float32))   # half-representable
    assert U.min() >= 0.0 and U.max() < 1.0
    assert abs(float(A.mean())) < 0.05 and abs(float(A.std()) - 1.0) < 0.05
    A2, U2 = synth.hash_draws(3, 4, 8, 50, seed=2)
    assert np.array_equal(A, A2) and np.array_equal(U, U2)
