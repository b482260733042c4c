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


def test_noalloc_index_sort_short_keys(mom):
    # K < 8: only the top K hash values are sorted and the common-prefix
    # count stops at K; compared with an index built with K = 3
    import torch
    wl = synth.tiny(43, n=5000, D=2, w=48, d=1, k=2, n_motifs=1)
    h = mom.Momenti(w=wl.w, d=wl.d, k=wl.k, delta=wl.delta, K=3, L=2,
                    precision=mom.PREC_FP32)
    h.hash_all(wl.series)
    M = h.info()["M"]
    for j, f in ((1, 1), (0, 0)):
        keys = np.ascontiguousarray(h.keys(j)[:, f])
        kt = torch.from_numpy(keys.view(np.int64)).cuda()
        order = torch.full((M,), -1, dtype=torch.int32, device="cuda")
        lcp = torch.full((M,), 255, dtype=torch.uint8, device="cuda")
        rc = mom.lib.momenti_index_sort_noalloc(C.c_void_p(kt.data_ptr()), M, 3,
                                                C.c_void_p(order.data_ptr()),
                                                C.c_void_p(lcp.data_ptr()), None)
        assert rc == mom.OK
        torch.cuda.synchronize()
        ref_order, ref_lcp = h.index(j, f)
        np.testing.assert_array_equal(order.cpu().numpy().view(np.uint32), ref_order)
        np.testing.assert_array_equal(lcp.cpu().numpy(), ref_lcp)
        assert int(lcp.max()) <= 3


def test_noalloc_index_sort_at_the_size_limit(mom):
    # exactly the largest accepted size (the scratch filled to the last
    # histogram tile), random keys with many shared leading bytes, against a
    # host stable sort and the common-prefix count written out on the host
    import torch
    m = mom.NOALLOC_MAX_KEYS
    rng = np.random.default_rng(7)
    hi = rng.integers(0, 4, size=m, dtype=np.uint64) << np.uint64(56)
    mid = rng.integers(0, 16, size=m, dtype=np.uint64) << np.uint64(40)
    lo = rng.integers(0, 1 << 20, size=m, dtype=np.uint64)
    keys = hi | mid | lo
    ref_order = np.argsort(keys, kind="stable").astype(np.uint32)
    srt = keys[ref_order]
    ref_lcp = np.zeros(m, dtype=np.uint8)
    for p in range(1, m):
        x = int(srt[p] ^ srt[p - 1])
        ref_lcp[p] = 8 if x == 0 else (63 - x.bit_length() + 1) // 8
    kt = torch.from_numpy(keys.view(np.int64)).cuda()
    for _ in range(2):
        order = torch.full((m,), -1, dtype=torch.int32, device="cuda")
        lcp = torch.full((m,), 255, dtype=torch.uint8, device="cuda")
        rc = mom.lib.momenti_index_sort_noalloc(C.c_void_p(kt.data_ptr()), m, 8,
                                                C.c_void_p(order.data_ptr()),
                                                C.c_void_p(lcp.data_ptr()), None)
        assert rc == mom.OK
        torch.cuda.synchronize()
        np.testing.assert_array_equal(order.cpu().numpy().view(np.uint32), ref_order)
        np.testing.assert_array_equal(lcp.cpu().numpy(), ref_lcp)
