"""The large memory-bounded form (D=64, w=1000, d=16, k=10, delta=0.01,
float32 random walk + sinusoids, twenty motifs planted in 16 dims each,
64 GB device-memory limit) through the C ABI.

* On its n = 2e5 prefix (the same generator at that length) the default
  search under the 64 GB limit returns the exact top-k that
  tests/golden/make_golden.py wrote with the oracle's C pair enumeration:
  pairs and dims identical, distances within 1e-9 relative.
* At full size (n = 1e7) the memory planner fits the index into the limit:
  the number of repetitions it chooses is reported, the device memory the
  handle takes stays below the limit, and the anytime search advances
  through its first repetitions, every current candidate carrying a miss
  bound in [0, 1].
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


def test_large_prefix_matches_the_exact_top_k(mom):
    gold = json.load(open(os.path.join(GOLDEN, "exact_large_form_n200000_seed0.json")))
    wl = synth.large_form(0, n=gold["n"])
    with mom.Momenti(w=wl.w, d=wl.d, k=wl.k, delta=wl.delta, mem_limit=wl.mem_limit) as h:
        h.hash_all(wl.series)
        got, st = h.topk()
    assert st["device_bytes"] <= wl.mem_limit
    ref = gold["motifs"]
    assert [(m["a"], m["b"]) for m in got] == [(m[1], m[2]) for m in ref]
    for g, r in zip(got, ref):
        assert g["dist_d"] == pytest.approx(r[0], rel=1e-9)
        assert g["dims"] == tuple(r[3])
        assert g["dist_max"] == pytest.approx(r[4], rel=1e-9)


def test_large_full_size_fits_the_memory_limit(mom):
    import torch
    wl = synth.large_form(0)
    x = torch.from_numpy(wl.series).cuda()
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    with mom.Momenti(w=wl.w, d=wl.d, k=wl.k, delta=wl.delta, mem_limit=wl.mem_limit) as h:
        h.hash_all(x)
        torch.cuda.synchronize()
        free1, _ = torch.cuda.mem_get_info()
        info = h.info()
        assert info["M"] == wl.n - wl.w + 1 and info["D"] == 64 and info["K"] == 8
        assert 1 <= info["L"]
        # the handle's allocations (index, scratch) stay inside the limit
        assert free0 - free1 <= wl.mem_limit
        h.search_begin()
        for _ in range(3):
            if h.search_step(1):
                break
        cur, (i, j, ended) = h.search_current()
        assert 1 <= i <= info["K"] and 0 <= j <= info["L"]
        for m in cur[wl.d]:
            assert 0.0 <= m["fail_bound"] <= 1.0
            assert len(m["dims"]) == wl.d
