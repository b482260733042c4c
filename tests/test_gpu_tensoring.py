"""Tensoring (Section 6.1) on the GPU, through the C ABI, against the
oracle's tensored keys and its Algorithm 1 with STOP on the re-derived
tensoring bound.

Half functions are passed explicitly: left function l at index 2 l, right
function r at 2 r + 1 (the layout of momenti_set_hash_params under
MOMENTI_FLAG_TENSORING); the oracle takes the same numbers as Al, Ar.

Tolerances: a tensored key is the interleave of one left and one right
half key, so each of its hash values must equal the oracle's except where
the exact (a . z + b) / r lies within the float32 band eta of an integer
(the bound of test_gpu_parity's hash test), where it may differ by one
bucket; top-k pairs and dims identical, distances within 1e-9 relative.
"""
import numpy as np
import pytest

from oracle import momenti_oracle as O
from paper_2502_14446_gb300 import synth

pytestmark = pytest.mark.gpu
U32 = 2.0 ** -24


@pytest.fixture(scope="module")
def mom():
    from paper_2502_14446_gb300 import build_ext
    build_ext.build()
    from paper_2502_14446_gb300 import momenti
    return momenti


def half_draws(D, m, K, w, seed):
    Al, Ul = synth.hash_draws(D, m, K // 2, w, seed)
    Ar, Ur = synth.hash_draws(D, m, K // 2, w, seed + 1000)
    A = np.empty((D, 2 * m, K // 2, w), np.float32)
    U = np.empty((D, 2 * m, K // 2), np.float32)
    A[:, 0::2], A[:, 1::2] = Al, Ar
    U[:, 0::2], U[:, 1::2] = Ul, Ur
    return A, U, (Al, Ul, Ar, Ur)


def make(mom, wl, m, K=8, r=0.0, seed=0, flags=0, precision=None, delta=None):
    A, U, lr = half_draws(wl.D, m, K, wl.w, seed)
    h = mom.Momenti(w=wl.w, d=wl.d, k=wl.k, delta=delta or wl.delta, K=K, L=m * m, r=r,
                    precision=mom.PREC_FP32 if precision is None else precision,
                    flags=mom.FLAG_TENSORING | flags)
    h.set_hash_params(A, U)
    h.hash_all(wl.series)
    return h, A, U, lr


def band(T, w, A, U, r, f):
    """(t, eta) of every (window, function, value) of dim f: the exact
    (a . z + b) / r and its float32 error band."""
    Z = O.znorm_windows(T[f], w)
    n_fn, Kh = A.shape[1], A.shape[2]
    absdot = np.abs(Z) @ np.abs(A[f].astype(np.float64)).reshape(-1, w).T
    v = Z @ A[f].astype(np.float64).reshape(-1, w).T
    b = (U[f].astype(np.float64) * r).reshape(-1)
    t = (v + b) / r
    eta = ((w + 8) * U32 * absdot + 4 * U32 * np.abs(v + b)) / r + 4 * U32 * np.abs(t)
    return t.reshape(-1, n_fn, Kh), (2 * eta).reshape(-1, n_fn, Kh)


@pytest.mark.parametrize("precision", ["fp32", "f16x2"])
def test_tensored_keys_match_the_oracle(mom, precision):
    wl = synth.tiny(31, 3000, 3, 64, 2, k=2, n_motifs=1)
    m, K = 4, 8
    prec = mom.PREC_FP32 if precision == "fp32" else mom.PREC_F16X2
    A, U, (Al, Ul, Ar, Ur) = half_draws(wl.D, m, K, wl.w, 31)
    r = O.estimate_r(wl.series, wl.w, Al)
    h, _, _, _ = make(mom, wl, m, K, r=r, seed=31, precision=prec)
    info = h.info()
    assert (info["L"], info["K"]) == (m * m, K)
    ref = O.tensored_keys(wl.series, wl.w, Al, Ul, Ar, Ur, r)             # (L, M, D)
    for f in range(wl.D):
        t, eta = band(wl.series, wl.w, A, U, r, f)                         # (M, 2m, K/2)
        sat = (t < -128) | (t >= 128)
        edge = (np.abs(t - np.round(t)) <= eta) & ~sat
        for jj in range(m * m):
            l, rr = divmod(jj, m)
            dev = h.keys(jj)[:, f]
            exp = ref[jj, :, f]
            for q in range(K):
                sh = np.uint64(56 - 8 * q)
                bd = ((dev >> sh) & np.uint64(255)).astype(np.int64)
                bo = ((exp >> sh) & np.uint64(255)).astype(np.int64)
                fn = 2 * l if q % 2 == 0 else 2 * rr + 1
                ok_edge = edge[:, fn, q // 2]
                diff = bd != bo
                assert not (diff & ~ok_edge).any(), (f, jj, q)
                assert (np.abs(bd - bo) <= 1).all()
    h.close()


def test_tensored_r_heuristic_uses_left_function_0(mom):
    wl = synth.tiny(32, 2500, 4, 50, 2, k=2, n_motifs=1)
    m = 3
    h, A, U, (Al, Ul, Ar, Ur) = make(mom, wl, m, seed=32)
    assert h.info()["r"] == pytest.approx(O.estimate_r(wl.series, wl.w, Al), rel=2e-5)
    a, u = h.hash_draws()
    np.testing.assert_array_equal(a, A[:, :2 * m])
    np.testing.assert_array_equal(u, U[:, :2 * m])
    h.close()


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_tensored_search_follows_the_oracle(mom, seed):
    # close planted motifs, m = 15 (L = 225), delta = 0.2: the oracle's
    # tensored Algorithm 1 stops on these seeds; the device result equals it,
    # and the oracle's traversal on the device's own keys stops where the
    # device stopped (whatever the keys), with the same bound
    wl = synth.tiny(seed, 1500, 3, 50, 2, k=2, n_motifs=2, noise=0.01)
    m, K, delta = 15, 8, 0.2
    A, U, (Al, Ul, Ar, Ur) = half_draws(wl.D, m, K, wl.w, seed)
    r = O.estimate_r(wl.series, wl.w, Al)
    h, _, _, _ = make(mom, wl, m, K, r=r, seed=seed, flags=mom.FLAG_NO_COST_SWITCH, delta=delta)
    got, st = h.topk()
    res = O.momenti_tensored(wl.series, wl.w, wl.d, wl.k, delta, Al, Ul, Ar, Ur, r)
    assert [(g["a"], g["b"]) for g in got] == [(x[1], x[2]) for x in res["motifs"]]
    for g, x in zip(got, res["motifs"]):
        assert g["dist_d"] == pytest.approx(x[0], rel=1e-9)
        assert g["dims"] == tuple(x[3])
    L = m * m
    keys_dev = np.stack([h.keys(j) for j in range(L)])
    Z = [O.znorm_windows(wl.series[f], wl.w) for f in range(wl.D)]

    def bound(dist_max, i, j):
        return O.tensoring_failure_bound(O.collision_probability(dist_max, r) ** wl.d, i, j, K, L)

    top, stop, _, _ = O.momenti_traverse(keys_dev, lambda a, b: O._pair_distances(Z, a, b),
                                         wl.d, wl.k, delta, r, O.exclusion_zone(wl.w), K,
                                         bound=bound)
    assert (st["stop_i"], st["stop_j"]) == (stop or (0, 0))
    if stop is not None:
        assert got[-1]["fail_bound"] == pytest.approx(bound(top[-1][4], *stop), rel=1e-3)
        assert got[-1]["fail_bound"] <= delta
    h.close()


def test_tensoring_keeps_L_a_square(mom):
    # L = 200 is not a square: the planner uses 14^2 = 196 repetitions,
    # drawn on the device as 28 half functions
    wl = synth.tiny(33, 1200, 2, 40, 1, k=1, n_motifs=1)
    with mom.Momenti(w=wl.w, d=wl.d, k=wl.k, delta=wl.delta, L=200,
                     flags=mom.FLAG_TENSORING) as h:
        h.hash_all(wl.series)
        assert h.info()["L"] == 196
        a, u = h.hash_draws()
        assert a.shape == (2, 28, 4, wl.w)
        got, st = h.topk()
        ref = O.exact_topk(wl.series, wl.w, wl.d, wl.k)
        if st["fallback"]:
            assert [(g["a"], g["b"]) for g in got] == [(x[1], x[2]) for x in ref]
