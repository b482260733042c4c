"""Robustness to irrelevant dimensions (Section 7, impact of noise): a
planted d-dimensional motif stays the returned top motif when 4 to 48
random-walk dimensions without motifs are added (recall 1 over the seeds),
and the result is the exact top-1 of the widened series."""
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


@pytest.mark.parametrize("extra", [4, 16, 48])
def test_planted_motif_survives_noise_dimensions(mom, extra):
    found = 0
    seeds = (1, 2, 3)
    for seed in seeds:
        base = synth.tiny(seed, 2000, 3, 50, 2, k=1, n_motifs=1, noise=0.02)
        wl = synth.with_noise_dims(base, extra, seed)
        a, b, dims = wl.planted[0]
        with mom.Momenti(w=wl.w, d=wl.d, k=1, delta=0.05) as h:
            h.hash_all(wl.series)
            got, st = h.topk()
        if (got[0]["a"], got[0]["b"]) == (a, b):
            found += 1
        ex = O.exact_topk(wl.series, wl.w, wl.d, 1)
        assert (got[0]["a"], got[0]["b"]) == (ex[0][1], ex[0][2])
        assert got[0]["dims"] == tuple(ex[0][3])
    assert found == len(seeds)
