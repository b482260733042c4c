"""The allocation-free index sort against the index momenti_hash_all builds.

Some callers cannot allocate device memory (they run under a fixed budget
reserved at start-up, or from inside another allocator); for them
momenti_index_sort_noalloc sorts one array of hash keys using only a fixed
scratch array compiled into the library.  Its order and common-prefix
lengths must equal those of the regular index, bit for bit, on two calls in
a row (the scratch keeps the previous call's contents).

This file is named to be collected last.
"""
import ctypes as C

import numpy as np
import pytest

from paper_2502_14446_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mom():
    from paper_2502_14446_gb300 import build_ext
    build_ext.build()
    from paper_2502_14446_gb300 import momenti
    return momenti


def test_noalloc_index_sort_equals_hash_all_index(mom):
    import torch
    wl = synth.tiny(41, n=6000, D=3, w=64, d=2, k=2, n_motifs=1)
    h = mom.Momenti(w=wl.w, d=wl.d, k=wl.k, delta=wl.delta, K=8, L=4,
                    precision=mom.PREC_FP32)
    h.hash_all(wl.series)
    M = h.info()["M"]
    stream = torch.cuda.current_stream().cuda_stream
    for j, f in ((0, 0), (3, 2)):              # two calls in a row
        keys = np.ascontiguousarray(h.keys(j)[:, f])
        kt = torch.from_numpy(keys.view(np.int64)).cuda()
        order = torch.full((M,), -1, dtype=torch.int32, device="cuda")
        lcp = torch.full((M,), 255, dtype=torch.uint8, device="cuda")
        rc = mom.lib.momenti_index_sort_noalloc(C.c_void_p(kt.data_ptr()), M, 8,
                                                C.c_void_p(order.data_ptr()),
                                                C.c_void_p(lcp.data_ptr()), C.c_void_p(stream))
        assert rc == mom.OK
        torch.cuda.synchronize()
        ref_order, ref_lcp = h.index(j, f)
        np.testing.assert_array_equal(order.cpu().numpy().view(np.uint32), ref_order)
        np.testing.assert_array_equal(lcp.cpu().numpy(), ref_lcp)


def test_noalloc_index_sort_rejects_oversize(mom):
    big = mom.NOALLOC_MAX_KEYS + 1
    rc = mom.lib.momenti_index_sort_noalloc(C.c_void_p(16), big, 8, C.c_void_p(16),
                                            C.c_void_p(16), None)
    assert rc == mom.ERR_OVERFLOW
