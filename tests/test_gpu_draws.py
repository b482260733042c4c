"""The hash functions drawn on the device (Eq. drp: a ~ N(0,1)^w, b = u r,
u ~ U[0,1)), read back through momenti_get_hash_draws.

The device generator is Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11).
This file writes the same generator from its published definition on the
host (checked against the publication's known-answer vectors) and compares
the device's integer stream through u bit for bit; the normals through
Box-Muller within one half-precision unit (the device evaluates log and
sincos in float32 before rounding to half); and the draws' distributions
by Kolmogorov-Smirnov tests against N(0,1) and U[0,1), moments,
half-representability of a and u < 1.
"""
import numpy as np
import pytest

from paper_2502_14446_gb300 import synth

M0, M1 = np.uint64(0xD2511F53), np.uint64(0xCD9E8D57)
W0, W1 = np.uint64(0x9E3779B9), np.uint64(0xBB67AE85)
MASK = np.uint64(0xFFFFFFFF)


def philox4x32_10(c0, c1, c2, c3, k0, k1):
    """Philox4x32 with 10 rounds on uint64 arrays holding 32-bit words:
    each round multiplies words 0 and 2 by M0 and M1, and the new counter is
    (hi(M1 c2) ^ c1 ^ k0, lo(M1 c2), hi(M0 c0) ^ c3 ^ k1, lo(M0 c0)); the key
    is bumped by the Weyl constants (W0, W1) between rounds."""
    c = [np.asarray(x, dtype=np.uint64) & MASK for x in (c0, c1, c2, c3)]
    k0 = np.asarray(k0, dtype=np.uint64) & MASK
    k1 = np.asarray(k1, dtype=np.uint64) & MASK
    for _ in range(10):
        p0 = M0 * c[0]
        p1 = M1 * c[2]
        c = [(p1 >> np.uint64(32)) ^ c[1] ^ k0, p1 & MASK, (p0 >> np.uint64(32)) ^ c[3] ^ k1,
             p0 & MASK]
        k0 = (k0 + W0) & MASK
        k1 = (k1 + W1) & MASK
    return c


def test_host_philox_known_answers():
    # known-answer vectors of the publication's reference implementation
    got = philox4x32_10(0, 0, 0, 0, 0, 0)
    assert [int(x) for x in got] == [0x6627E8D5, 0xE169C58D, 0xBC57AC4C, 0x9B00DBD8]
    f = 0xFFFFFFFF
    got = philox4x32_10(f, f, f, f, f, f)
    assert [int(x) for x in got] == [0x408F276D, 0x41C83B0E, 0xA20BC7C6, 0x6D5451FD]
    got = philox4x32_10(0x243F6A88, 0x85A308D3, 0x13198A2E, 0x03707344, 0xA4093822, 0x299F31D0)
    assert [int(x) for x in got] == [0xD16CFE09, 0x94FDCCEB, 0x5001E420, 0x24126EA1]


def host_draws(seed, count_a, count_u):
    """The documented stream: u = (x >> 8) 2^-24 from stream 1; a from
    Box-Muller on stream 0 (float64 here), rounded to half."""
    qa = np.arange((count_a + 3) // 4, dtype=np.uint64)
    ra = philox4x32_10(qa, qa >> np.uint64(32), 0, 0, seed & 0xFFFFFFFF, seed >> 32)
    z = np.empty((qa.size, 4))
    for h in range(2):
        u1 = ((ra[2 * h] >> np.uint64(8)) + np.uint64(1)).astype(np.float64) * 2.0 ** -24
        u2 = (ra[2 * h + 1] >> np.uint64(8)).astype(np.float64) * 2.0 ** -24
        rad = np.sqrt(-2.0 * np.log(u1))
        z[:, 2 * h] = rad * np.cos(2 * np.pi * u2)
        z[:, 2 * h + 1] = rad * np.sin(2 * np.pi * u2)
    a = z.reshape(-1)[:count_a]
    qu = np.arange((count_u + 3) // 4, dtype=np.uint64)
    ru = philox4x32_10(qu, qu >> np.uint64(32), 1, 0, seed & 0xFFFFFFFF, seed >> 32)
    u = np.stack([(x >> np.uint64(8)).astype(np.float64) * 2.0 ** -24 for x in ru], 1)
    return a, u.reshape(-1)[:count_u]


@pytest.fixture(scope="module")
def drawn():
    from paper_2502_14446_gb300 import build_ext
    build_ext.build()
    from paper_2502_14446_gb300 import momenti
    wl = synth.tiny(3, n=2000, D=8, w=64, d=2, k=2, n_motifs=0)
    seed = 0x1234_5678_9ABC
    with momenti.Momenti(w=wl.w, d=wl.d, k=wl.k, delta=wl.delta, K=8, L=200, seed=seed,
                         precision=momenti.PREC_FP32) as h:
        h.hash_all(wl.series)
        a, u = h.hash_draws()
    assert a.shape == (8, 200, 8, 64) and u.shape == (8, 200, 8)
    return seed, a.reshape(-1), u.reshape(-1)


@pytest.mark.gpu
def test_device_uniforms_are_the_philox_stream(drawn):
    seed, a, u = drawn
    _, u_ref = host_draws(seed, 4, u.size)
    np.testing.assert_array_equal(u.astype(np.float64), u_ref)
    assert u.min() >= 0.0 and u.max() < 1.0


@pytest.mark.gpu
def test_device_normals_follow_box_muller_on_the_stream(drawn):
    seed, a, u = drawn
    a_ref, _ = host_draws(seed, a.size, 4)
    # a is half-representable: rounding to half again changes nothing
    np.testing.assert_array_equal(a.astype(np.float16).astype(np.float32), a)
    ref_half = a_ref.astype(np.float16).astype(np.float64)
    diff = np.abs(a.astype(np.float64) - ref_half)
    # one half-precision unit at the value's magnitude (normal range, |a| >= 2^-14)
    ulp = 2.0 ** (np.floor(np.log2(np.maximum(np.abs(ref_half), 2.0 ** -14))) - 10)
    assert np.all(diff <= ulp * 1.0000001)
    assert (diff == 0).mean() > 0.99


@pytest.mark.gpu
def test_device_draws_are_distributed_as_eq_drp_requires(drawn):
    from scipy import stats
    _, a, u = drawn
    a = a.astype(np.float64)
    n = a.size
    assert abs(a.mean()) < 5.0 / np.sqrt(n)
    assert abs(a.var() - 1.0) < 5.0 * np.sqrt(2.0 / n)
    assert abs(stats.skew(a)) < 5.0 * np.sqrt(6.0 / n)
    assert stats.kstest(a, "norm").pvalue > 1e-3
    assert stats.kstest(u.astype(np.float64), "uniform").pvalue > 1e-3
    # different (f, j, k) functions are not copies of one another
    rows = a.reshape(-1, 64)
    assert np.unique(rows[:, :4], axis=0).shape[0] == rows.shape[0]
