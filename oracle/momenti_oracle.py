"""CPU oracle for the LSH top-k multidimensional motif search (MOMENTI,
arXiv 2502.14446).

TEST INFRASTRUCTURE ONLY.  Nothing on the product path may import, call or
execute this module: only the tests, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg use it.  It shares no code with the CUDA
library; the two meet only through the seeded inputs of
``paper_2502_14446_gb300.synth``.

Everything is float64 numpy, written to be read against the paper:

* Section 3.1: the z-normalised Euclidean distance (Eq. zned) with the
  population standard deviation, the d-dimensional distance ``dist_d``
  (Definition distdims), ``dims_d``, ``dist_d^max`` (Eq. distdmax), trivial
  matches with exclusion zone ``eps = w/2`` and the top-k motif set.
* Section 3.2: the discretised random projection hash (Eq. drp), its
  collision probability (Eq. eucl-collision-probability), concatenation K and
  repetitions L.
* Algorithm 1 (MOMENTI) and Algorithm 2 (STOP), in the paper's loop order.
* Section 6.1: the heuristic for the quantisation width r, and tensoring:
  interleaved keys, a re-derived miss-probability bound, and Algorithm 1
  with STOP on that bound.
* Section 6.3: motifs of several dimensionalities in one traversal.

Readings of points the paper leaves open (each is listed with its reason in
the design notes of the repository):

* sigma is the population standard deviation (so dist lies in [0, 2 sqrt(w)]
  and dist^2 = 2w(1 - corr), Section 2);
* a window whose sigma is at most ``FLAT_REL * (1 + |mu|)`` is flat: its
  z-normalised form is the zero vector;
* trivial match iff ``|a - b| <= eps`` with ``eps = floor(w / 2)``;
* the top-k set is built greedily in ascending (dist_d, a, b) order, a pair
  being accepted iff none of its two indices is within eps of an index of an
  already accepted pair (the matrix-profile procedure of Section 2);
* TOP of Algorithm 1 is that greedy selection over every distinct pair
  verified so far; TOP.max() is its k-th pair;
* a hash value is floor((a . z + b) / r) of the z-normalised window z,
  saturated to a signed byte; a composite key packs the K bytes big-endian,
  concatenation 0 in the most significant byte, byte value h + 128;
* r is (max - min) / 256 over projections of evenly spaced sample windows
  onto the K vectors of repetition 0 of every dimension.

Every function here is pinned, directly or through the function that uses
it, by the tests of tests/test_oracle.py (and the stored records by
tests/test_golden.py) against the paper or the mathematics: closed forms,
brute force on tiny inputs, Monte Carlo, hand-evaluated tables, and the
printed example of Section 4.  No function is unpinned.
"""
from __future__ import annotations

import itertools
import math

import numpy as np

FLAT_REL = 1e-8          # flat-window threshold, relative to 1 + |mu|
R_BUCKETS = 256          # Section 6.1: 256 equal-width buckets, one byte per value
R_SAMPLE_WINDOWS = 4096  # sample windows per dimension for the r heuristic


# ---------------------------------------------------------------------------
# Section 3.1: distances
# ---------------------------------------------------------------------------

def exclusion_zone(w: int, excl: int | None = None) -> int:
    """Trivial-match exclusion zone eps (Section 3.1: eps = w/2)."""
    return int(w // 2) if excl is None or excl < 0 else int(excl)


def window_stats(x: np.ndarray, w: int):
    """Mean and population standard deviation of every length-w window of a
    one-dimensional series, by the two-pass formula (Eq. zned's mu, sigma).
    Returns (mu, sigma, flat) arrays of length n - w + 1."""
    x = np.asarray(x, dtype=np.float64)
    V = np.lib.stride_tricks.sliding_window_view(x, w)
    mu = V.mean(axis=1)
    sigma = np.sqrt(((V - mu[:, None]) ** 2).mean(axis=1))
    flat = sigma <= FLAT_REL * (1.0 + np.abs(mu))
    return mu, sigma, flat


def znorm_windows(x: np.ndarray, w: int) -> np.ndarray:
    """All z-normalised windows of a one-dimensional series, shape (M, w);
    flat windows map to the zero vector."""
    x = np.asarray(x, dtype=np.float64)
    V = np.lib.stride_tricks.sliding_window_view(x, w)
    mu, sigma, flat = window_stats(x, w)
    s = np.where(flat, 1.0, sigma)
    Z = (V - mu[:, None]) / s[:, None]
    Z[flat] = 0.0
    return Z


def zned(u: np.ndarray, v: np.ndarray) -> float:
    """Eq. (zned): z-normalised Euclidean distance of two equal-length
    windows, population sigma, flat windows normalised to zero."""
    u = np.asarray(u, dtype=np.float64)
    v = np.asarray(v, dtype=np.float64)

    def z(x):
        mu = x.mean()
        sd = math.sqrt(((x - mu) ** 2).mean())
        if sd <= FLAT_REL * (1.0 + abs(mu)):
            return np.zeros_like(x)
        return (x - mu) / sd

    return float(math.sqrt(((z(u) - z(v)) ** 2).sum()))


def per_dim_distances(T: np.ndarray, w: int, a: int, b: int) -> np.ndarray:
    """dist(T_a^f, T_b^f) for every dimension f (Eq. zned per dimension)."""
    return np.array([zned(T[f, a:a + w], T[f, b:b + w]) for f in range(T.shape[0])])


def select_d(dists: np.ndarray, d: int):
    """Definition distdims / Eq. distdmax on one pair's per-dimension
    distances: returns (dist_d, dims_d, dist_d^max).  dist_d is the sum of
    the d smallest distances (the minimum over all size-d subsets); ties go
    to the lower dimension index."""
    order = np.argsort(np.asarray(dists, dtype=np.float64), kind="stable")[:d]
    dims = tuple(sorted(int(f) for f in order))
    vals = np.asarray(dists, dtype=np.float64)[list(dims)]
    return float(vals.sum()), dims, float(vals.max())


def dims_mask(dims) -> int:
    m = 0
    for f in dims:
        m |= 1 << int(f)
    return m


# ---------------------------------------------------------------------------
# top-k under the trivial-match exclusion
# ---------------------------------------------------------------------------

def greedy_topk(cands, k: int, eps: int):
    """Top-k motif set of Section 3.1 from candidate pairs.

    ``cands`` is an iterable of (dist_d, a, b, payload) with a < b.  Pairs
    are taken in ascending (dist_d, a, b) order and a pair is accepted iff
    b - a > eps and both of its indices are more than eps away from both
    indices of every accepted pair.  Returns the accepted tuples."""
    acc = []
    for c in sorted(cands, key=lambda t: (t[0], t[1], t[2])):
        _, a, b = c[0], c[1], c[2]
        if b - a <= eps:
            continue
        ok = True
        for q in acc:
            for x in (a, b):
                for y in (q[1], q[2]):
                    if abs(x - y) <= eps:
                        ok = False
        if ok:
            acc.append(c)
            if len(acc) == k:
                break
    return acc


def naive_topk(T: np.ndarray, w: int, d: int, k: int, excl: int | None = None):
    """Top-k d-dimensional motifs by plain enumeration of the definitions:
    every pair of windows, Eq. (zned) per dimension, the minimum of the sum
    over every size-d subset of dimensions (Definition distdims).  Only for
    tiny inputs.  Returns [(dist_d, a, b, dims, dist_max)]."""
    T = np.asarray(T, dtype=np.float64)
    D, n = T.shape
    M = n - w + 1
    eps = exclusion_zone(w, excl)
    subsets = list(itertools.combinations(range(D), d))
    cands = []
    for a in range(M):
        for b in range(a + eps + 1, M):
            dist = per_dim_distances(T, w, a, b)
            best = None
            for F in subsets:
                s = float(sum(dist[f] for f in F))
                if best is None or s < best[0]:
                    best = (s, F)
            F = best[1]
            cands.append((best[0], a, b, (tuple(F), float(max(dist[f] for f in F)))))
    out = greedy_topk(cands, k, eps)
    return [(c[0], c[1], c[2], c[3][0], c[3][1]) for c in out]


def _pair_distances(Z: list, a: np.ndarray, b: np.ndarray) -> np.ndarray:
    """Per-dimension distances of many pairs from z-normalised windows:
    sqrt(sum_t (z_a[t] - z_b[t])^2), shape (D, m)."""
    out = np.empty((len(Z), a.size))
    for f, Zf in enumerate(Z):
        diff = Zf[a] - Zf[b]
        out[f] = np.sqrt((diff * diff).sum(axis=1))
    return out


def _select_d_many(dist: np.ndarray, d: int):
    """select_d over the columns of a (D, m) distance array."""
    order = np.argsort(dist, axis=0, kind="stable")[:d]
    order.sort(axis=0)
    vals = np.take_along_axis(dist, order, axis=0)
    masks = np.zeros(dist.shape[1], dtype=np.uint64)
    for r in range(d):
        masks |= np.left_shift(np.uint64(1), order[r].astype(np.uint64))
    return vals.sum(axis=0), masks, vals.max(axis=0), order


def exact_topk(T: np.ndarray, w: int, d: int, k: int, excl: int | None = None,
               tau: float = math.inf, block: int = 512):
    """Exact top-k d-dimensional motifs over all pairs (the quantity
    Algorithm 1 returns with probability >= 1 - delta, and what its last
    line computes when STOP never holds).

    Per dimension, dist^2 = |z_a|^2 + |z_b|^2 - 2 z_a . z_b, the expanded
    square of Eq. (zned) (the Pearson form of Section 2) with a library
    matrix product for the dot products, enumerated in blocks of rows.
    dist_d is the sum of the d smallest per-dimension distances.  Pairs with
    dist_d > tau are not collected (tau = inf keeps all; a pair can only
    have dist_d <= tau if at least d of its dimensions are <= tau).
    Returns [(dist_d, a, b, dims, dist_max)] or None if fewer than k pairs
    could be selected below tau."""
    T = np.asarray(T, dtype=np.float64)
    D, n = T.shape
    M = n - w + 1
    eps = exclusion_zone(w, excl)
    Z = [znorm_windows(T[f], w) for f in range(D)]
    nrm = [(Zf * Zf).sum(axis=1) for Zf in Z]
    cand_a, cand_b, cand_dist = [], [], []
    for a0 in range(0, M, block):
        a1 = min(M, a0 + block)
        rows = np.arange(a0, a1)
        dist = np.empty((D, a1 - a0, M))
        for f in range(D):
            G = Z[f][a0:a1] @ Z[f].T
            sq = nrm[f][a0:a1, None] + nrm[f][None, :] - 2.0 * G
            dist[f] = np.sqrt(np.maximum(sq, 0.0))
        valid = (np.arange(M)[None, :] - rows[:, None]) > eps
        if math.isfinite(tau):
            valid &= (dist <= tau).sum(axis=0) >= d
        ia, ib = np.nonzero(valid)
        if ia.size == 0:
            continue
        sel = dist[:, ia, ib]
        dd = np.sort(sel, axis=0)[:d].sum(axis=0)
        keep = dd <= tau
        cand_a.append(ia[keep] + a0)
        cand_b.append(ib[keep])
        cand_dist.append(sel[:, keep])
    if not cand_a:
        return None
    A = np.concatenate(cand_a)
    B = np.concatenate(cand_b)
    dist = np.concatenate(cand_dist, axis=1)
    dd, masks, dmax, order = _select_d_many(dist, d)
    idx = np.lexsort((B, A, dd))
    # greedy selection of Section 3.1 over the sorted candidates
    acc = []
    for t in idx:
        a, b = int(A[t]), int(B[t])
        ok = True
        for q in acc:
            if (abs(a - q[1]) <= eps or abs(a - q[2]) <= eps
                    or abs(b - q[1]) <= eps or abs(b - q[2]) <= eps):
                ok = False
                break
        if ok:
            acc.append((float(dd[t]), a, b, tuple(int(f) for f in order[:, t]), float(dmax[t])))
            if len(acc) == k:
                break
    if len(acc) < k:
        return None
    return acc


_PAIR = np.dtype([("a", np.int64), ("b", np.int64), ("dist_d", np.float64),
                  ("dist_max", np.float64), ("dims", np.uint64)])
_CLIB = None


def _pairs_lib():
    """The oracle's C pair enumeration (exact_pairs.c), built on first use."""
    global _CLIB
    if _CLIB is None:
        import ctypes as C
        from oracle import build_c
        lib = C.CDLL(build_c.build())
        fn = lib.oracle_pairs_below
        fn.restype = C.c_int64
        fn.argtypes = [C.c_void_p, C.c_int, C.c_int64, C.c_int, C.c_int, C.c_int64, C.c_double,
                       C.c_double, C.c_void_p, C.c_int64]
        _CLIB = fn
    return _CLIB


def pairs_below(T: np.ndarray, w: int, d: int, tau: float, excl: int | None = None) -> np.ndarray:
    """Every non-trivial pair (b - a > eps) with dist_d <= tau, as a record
    array (a, b, dist_d, dist_max, dims mask), sorted by (dist_d, a, b).
    Computed by exact_pairs.c: float64 sliding dot products along the
    diagonals (recomputed directly every 1024 steps) in the Pearson form of
    Eq. zned, the d smallest per-dimension distances (ties to the lower
    dimension), flat windows as in znorm_windows."""
    import ctypes as C
    T = np.ascontiguousarray(T, dtype=np.float64)
    D, n = T.shape
    eps = exclusion_zone(w, excl)
    cap = 1 << 16
    while True:
        out = np.zeros(cap, dtype=_PAIR)
        cnt = _pairs_lib()(T.ctypes.data_as(C.c_void_p), D, n, w, d, eps, float(tau), FLAT_REL,
                           out.ctypes.data_as(C.c_void_p), cap)
        if cnt < 0:
            raise MemoryError("exact_pairs: out of memory")
        if cnt <= cap:
            out = out[:cnt]
            return out[np.lexsort((out["b"], out["a"], out["dist_d"]))]
        cap = 1 << int(cnt - 1).bit_length()


def exact_topk_diag(T, w, d, k, excl=None, tau0: float = 1.0):
    """The exact top-k (same quantity and record format as exact_topk) from
    pairs_below: collect every pair with dist_d <= tau, select greedily in
    (dist_d, a, b) order, and double tau until k pairs are selected with
    the k-th at or below tau (then no unseen pair can change the
    selection).  Fewer than k are returned only when tau covers every pair
    (2 d sqrt(w), the largest possible dist_d).

    The sliding recurrence of pairs_below carries float64 rounding drift
    (about 1e-9 relative), so it only picks the candidates: every pair up
    to just past the k-th selected one (1e-6 relative, far above the drift)
    is evaluated again by the definition (Eq. zned per dimension, direct
    sums) and the greedy selection runs on those values."""
    eps = exclusion_zone(w, excl)
    T64 = np.ascontiguousarray(T, dtype=np.float64)
    tau = float(tau0)
    top = 2.0 * d * math.sqrt(w)
    while True:
        cands = pairs_below(T, w, d, tau, excl)
        rough = greedy_topk([(float(c["dist_d"]), int(c["a"]), int(c["b"])) for c in cands], k, eps)
        edge = tau if len(rough) < k else rough[-1][0] * (1.0 + 1e-6) + 1e-9
        exact = []
        for c in cands:
            if float(c["dist_d"]) > edge:
                break
            a, b = int(c["a"]), int(c["b"])
            dd, dims, dmax = select_d(per_dim_distances(T64, w, a, b), d)
            exact.append((dd, a, b, dims, dmax))
        acc = greedy_topk(exact, k, eps)
        if (len(acc) == k and acc[-1][0] <= tau) or tau >= top:
            return acc
        tau *= 2.0


def exact_topk_auto(T, w, d, k, excl=None, tau0: float | None = None, block: int = 512):
    """exact_topk with tau doubled until k pairs are selected (tau0 = None
    means no threshold)."""
    if tau0 is None:
        return exact_topk(T, w, d, k, excl, math.inf, block)
    tau = tau0
    while True:
        res = exact_topk(T, w, d, k, excl, tau, block)
        if res is not None and res[-1][0] <= tau:
            return res
        tau *= 2.0


# ---------------------------------------------------------------------------
# Section 3.2: the hash family and its collision probability
# ---------------------------------------------------------------------------

def std_normal_cdf(x: float) -> float:
    return 0.5 * math.erfc(-x / math.sqrt(2.0))


def collision_probability(R: float, r: float) -> float:
    """Eq. (eucl-collision-probability): Pr[h(x) = h(y)] for two vectors at
    Euclidean distance R under h(x) = floor((a.x + b)/r)."""
    if R <= 0.0:
        return 1.0
    c = r / R
    return (1.0 - 2.0 * std_normal_cdf(-c)
            - 2.0 / (math.sqrt(2.0 * math.pi) * c) * (1.0 - math.exp(-c * c / 2.0)))


def stop_condition(dist_max: float, i: int, j: int, K: int, L: int, d: int,
                   delta: float, r: float) -> bool:
    """Algorithm 2: p = P(dist_d^max)^d; at i = K stop iff (1 - p^i)^j <= delta,
    otherwise iff (1 - p^i)^j (1 - p^(i+1))^(L-j) <= delta.  i and j are
    1-based, as in Algorithm 1."""
    return failure_bound(dist_max, i, j, K, L, d, r) <= delta


def failure_bound(dist_max: float, i: int, j: int, K: int, L: int, d: int, r: float) -> float:
    """The miss-probability bound of Lemma stop (Eq. probnotcolliding)."""
    p = collision_probability(dist_max, r) ** d
    if i == K:
        return (1.0 - p ** i) ** j
    return (1.0 - p ** i) ** j * (1.0 - p ** (i + 1)) ** (L - j)


def tensoring_failure_bound(p: float, i: int, j: int, K: int, L: int) -> float:
    """Miss probability of a pair under tensoring (Section 6.1), re-derived.

    Tensoring builds repetition j (0-based j' = j - 1 -> left function
    l = j' div m, right function r = j' mod m, m = sqrt(L)) from m left and
    m right functions of K/2 concatenated hashes each; the composite key
    interleaves them (left value first), so a prefix of length t collides
    iff the left prefix of ceil(t/2) values and the right prefix of
    floor(t/2) values both collide.  ``p`` is the probability that one
    hash function collides in all d dims of the pair (the caller passes
    P(dist_max)^d, a lower bound, as in Lemma stop); the K/2 values of one
    function collide independently, so the collision depth G of a function
    has P(G >= u) = p^u, and all 2m functions are independent.

    After j repetitions at prefix length i, every repetition has been seen
    at length i + 1 (i < K), the first j also at length i.  The pair was
    missed iff no visited (repetition, length) collides.  Rows l and
    columns r fall into groups that are visited alike (rows before the
    current one, the current one, rows after it; columns before the
    current one and the rest), and within a pair of groups every
    (row, column) combination is visited, so only the largest depth class
    of each group matters: the result sums over those classes exactly.
    The miss probability decreases as p grows, so a lower bound on p gives
    an upper bound.  Needs L = m^2, K even, 1 <= i <= K, 0 <= j <= L."""
    if L < 1:
        raise ValueError("tensoring needs L = m^2 >= 1")
    m = math.isqrt(L)
    if m * m != L or K % 2 or not 1 <= i <= K or not 0 <= j <= L:
        raise ValueError("tensoring needs L = m^2, K even, 1 <= i <= K, 0 <= j <= L")
    top = i == K
    # depth thresholds: length i and length i + 1, rows (left) and columns (right)
    ug = (-(-i // 2), -(-(i + 1) // 2) if not top else -(-i // 2))
    uh = (i // 2, (i + 1) // 2 if not top else i // 2)

    def class_probs(u):
        # class 0: depth < u[0]; 1: u[0] <= depth < u[1]; 2: depth >= u[1]
        s1, s2 = p ** u[0], p ** u[1]
        return [1.0 - s1, s1 - s2, s2]

    def max_class_probs(cp, size):
        # distribution of the largest class among `size` iid rows (-1: none)
        if size == 0:
            return {-1: 1.0}
        cdf = np.cumsum(cp)
        out, prev = {}, 0.0
        for c in range(3):
            cur = min(1.0, cdf[c]) ** size
            out[c] = cur - prev
            prev = cur
        return out

    a, b = divmod(j, m)
    rows = [a, 1 if a < m else 0, max(0, m - a - 1)]     # before, current, after
    cols = [b, m - b]                                     # before the current, the rest
    # (row group, column group, 0 = length i / 1 = length i + 1) visited
    visits = [(0, 0, 0), (0, 1, 0), (1, 0, 0)]
    if not top:
        visits += [(1, 1, 1), (2, 0, 1), (2, 1, 1)]
    gdist = [max_class_probs(class_probs(ug), n) for n in rows]
    hdist = [max_class_probs(class_probs(uh), n) for n in cols]
    miss = 0.0
    for g0, pg0 in gdist[0].items():
        for g1, pg1 in gdist[1].items():
            for g2, pg2 in gdist[2].items():
                gm = (g0, g1, g2)
                for h0, ph0 in hdist[0].items():
                    for h1, ph1 in hdist[1].items():
                        hm = (h0, h1)
                        # a visit at length i needs class >= 1 on both
                        # sides, at length i + 1 class 2 on both
                        hit = any(gm[rg] >= 1 + lv and hm[cg] >= 1 + lv for rg, cg, lv in visits)
                        if not hit:
                            miss += pg0 * pg1 * pg2 * ph0 * ph1
    return float(miss)


def projections(T: np.ndarray, w: int, A: np.ndarray, f: int, windows=None) -> np.ndarray:
    """a . z for z-normalised windows of dimension f and vectors A (..., w).
    Returns shape (len(windows), prod(A.shape[:-1]))."""
    Z = znorm_windows(T[f], w)
    if windows is not None:
        Z = Z[windows]
    return Z @ np.asarray(A, dtype=np.float64).reshape(-1, w).T


def estimate_r(T: np.ndarray, w: int, A: np.ndarray, samples: int = R_SAMPLE_WINDOWS) -> float:
    """Section 6.1 heuristic: project sample windows on random Gaussian
    vectors, split the observed range into 256 equal-width buckets and use
    the bucket width as r.  The sample is min(M, samples) evenly spaced
    windows per dimension; the vectors are the K vectors of repetition 0 of
    each dimension (A has shape (D, L, K, w)); the range is pooled over all
    dimensions."""
    T = np.asarray(T, dtype=np.float64)
    D, n = T.shape
    M = n - w + 1
    S = min(M, samples)
    pos = sample_positions(M, S)
    lo, hi = math.inf, -math.inf
    for f in range(D):
        v = projections(T, w, A[f, 0], f, pos)
        lo = min(lo, float(v.min()))
        hi = max(hi, float(v.max()))
    if not hi > lo:
        return 1.0
    return (hi - lo) / R_BUCKETS


def sample_positions(M: int, S: int) -> np.ndarray:
    """Evenly spaced window positions: floor(q * (M - 1) / (S - 1)), q < S."""
    if S <= 1:
        return np.zeros(1, dtype=np.int64)
    q = np.arange(S, dtype=np.int64)
    return (q * (M - 1)) // (S - 1)


def hash_values(T: np.ndarray, w: int, A: np.ndarray, U: np.ndarray, r: float, f: int):
    """Eq. (drp) for every window of dimension f and every (j, k):
    t = (a . z + b) / r with b = U r, h = floor(t) saturated to [-128, 127].
    Returns (h int16 (M, L, K), t float64 (M, L, K))."""
    L, K, w_ = A.shape[1:]
    assert w_ == w
    v = projections(T, w, A[f], f).reshape(-1, L, K)
    b = U[f].astype(np.float64) * r
    t = (v + b[None]) / r
    h = np.clip(np.floor(t), -128, 127).astype(np.int16)
    return h, t


def pack_keys(h: np.ndarray) -> np.ndarray:
    """Pack K hash bytes into one uint64, big-endian: concatenation 0 in the
    most significant byte, byte value h + 128 (h saturated to a signed
    byte).  Lexicographic order of keys is the order of the hash strings
    (Section 4, index construction).  h has shape (..., K)."""
    K = h.shape[-1]
    key = np.zeros(h.shape[:-1], dtype=np.uint64)
    for kk in range(K):
        byte = (h[..., kk].astype(np.int64) + 128).astype(np.uint64)
        key |= np.left_shift(byte, np.uint64(56 - 8 * kk))
    return key


def hash_all(T: np.ndarray, w: int, A: np.ndarray, U: np.ndarray, r: float):
    """Algorithm 1, initialisation: the composite hash h_{K,j}^f of every
    window, dimension and repetition.  Returns (keys uint64 (L, M, D),
    t float64 (D, M, L, K))."""
    T = np.asarray(T, dtype=np.float64)
    D = T.shape[0]
    L, K = A.shape[1], A.shape[2]
    M = T.shape[1] - w + 1
    keys = np.empty((L, M, D), dtype=np.uint64)
    ts = np.empty((D, M, L, K))
    for f in range(D):
        h, t = hash_values(T, w, A, U, r, f)
        keys[:, :, f] = pack_keys(h).T
        ts[f] = t
    return keys, ts


def prefix(key, i: int):
    """h_{i,j}: the first i hash values of a composite key."""
    return np.right_shift(np.asarray(key, dtype=np.uint64), np.uint64(64 - 8 * i))


def build_index(keys: np.ndarray):
    """Section 4, index construction: for every (j, f) the windows in
    lexicographic order of their hash strings (ties by window index), plus
    the length of the common prefix (in hash values) of each entry with the
    previous one.  Returns (order uint32 (L, D, M), lcp uint8 (L, D, M))."""
    L, M, D = keys.shape
    order = np.empty((L, D, M), dtype=np.uint32)
    lcp = np.zeros((L, D, M), dtype=np.uint8)
    for j in range(L):
        for f in range(D):
            o = np.argsort(keys[j, :, f], kind="stable")
            order[j, f] = o
            s = keys[j, o, f]
            for p in range(1, M):
                x = int(s[p - 1]) ^ int(s[p])
                lcp[j, f, p] = 8 if x == 0 else (64 - x.bit_length()) // 8
    return order, lcp


# ---------------------------------------------------------------------------
# Algorithm 1 and Algorithm 2
# ---------------------------------------------------------------------------

def colliding_pairs(keys_jf: np.ndarray, i: int) -> np.ndarray:
    """Collision step of Algorithm 1: all pairs (a < b) whose hash strings share the
    prefix of length i, for one (j, f).  Returns codes a * M + b (int64)."""
    M = keys_jf.size
    pre = prefix(keys_jf, i)
    uniq, inv, cnt = np.unique(pre, return_inverse=True, return_counts=True)
    out = []
    for g in np.nonzero(cnt >= 2)[0]:
        members = np.sort(np.nonzero(inv == g)[0]).astype(np.int64)
        ia, ib = np.triu_indices(members.size, 1)
        out.append(members[ia] * M + members[ib])
    if not out:
        return np.zeros(0, dtype=np.int64)
    return np.concatenate(out)


class _Pool:
    """Every distinct verified pair, with the greedy TOP selection.

    The greedy selection only changes when a new pair is closer than the
    current k-th selected pair (pairs further away are visited after the
    k-th acceptance), so it is recomputed only then."""

    def __init__(self, k: int, eps: int):
        self.k, self.eps = k, eps
        self.pairs = {}
        self._top = []

    def add_many(self, a, b, dd, order, dmax):
        kth = self._top[-1][0] if len(self._top) == self.k else math.inf
        dirty = False
        for t in range(len(a)):
            key = (int(a[t]), int(b[t]))
            if key in self.pairs:
                continue
            self.pairs[key] = (float(dd[t]), tuple(int(f) for f in order[:, t]), float(dmax[t]))
            if float(dd[t]) <= kth:
                dirty = True
        if dirty:
            cands = [(v[0], a_, b_, (v[1], v[2])) for (a_, b_), v in self.pairs.items()]
            sel = greedy_topk(cands, self.k, self.eps)
            self._top = [(c[0], c[1], c[2], c[3][0], c[3][1]) for c in sel]

    def top(self):
        return list(self._top)


def momenti_traverse(keys: np.ndarray, pair_distances, d: int, k: int, delta: float,
                     r: float, eps: int, K: int | None = None, bound=None):
    """The prefix traversal of Algorithm 1 over given composite hash keys
    (uint64, shape (L, M, D)): for i = K..1, for j = 1..L, W(a, b) counts the
    dimensions in which a and b share the length-i prefix; every pair with
    W >= d that is not a trivial match is verified with
    ``pair_distances(a, b) -> (D, m)`` and offered to TOP; the loop returns
    when |TOP| = k and STOP(TOP.max(), i, j, delta) (Algorithm 2).

    ``bound(dist_max, i, j)``, when given, replaces Lemma stop's bound in
    the STOP test (tensoring).

    Returns (top, (i, j) or None, n_dist, pool_size)."""
    L, M, D = keys.shape
    K = 8 if K is None else K
    pool = _Pool(k, eps)
    n_dist = 0
    for i in range(K, 0, -1):
        for j in range(1, L + 1):
            codes = [colliding_pairs(keys[j - 1, :, f], i) for f in range(D)]
            allc = np.concatenate(codes) if codes else np.zeros(0, np.int64)
            uniq, W = np.unique(allc, return_counts=True)
            sel = uniq[W >= d]
            a = sel // M
            b = sel % M
            nt = (b - a) > eps
            a, b = a[nt], b[nt]
            if a.size:
                dist = pair_distances(a, b)
                n_dist += int(a.size)
                dd, masks, dmax, order = _select_d_many(dist, d)
                pool.add_many(a, b, dd, order, dmax)
            top = pool.top()
            if len(top) == k:
                done = (stop_condition(top[-1][4], i, j, K, L, d, delta, r) if bound is None
                        else bound(top[-1][4], i, j) <= delta)
                if done:
                    return top, (i, j), n_dist, len(pool.pairs)
    return None, None, n_dist, len(pool.pairs)


def momenti(T: np.ndarray, w: int, d: int, k: int, delta: float, A: np.ndarray,
            U: np.ndarray, r: float, excl: int | None = None, all_k: bool = False,
            fallback_tau: float | None = None):
    """Algorithm 1 (MOMENTI) with Algorithm 2 (STOP), in the paper's order:
    hash every window, dimension and repetition, traverse the prefixes
    (``momenti_traverse``) and, if STOP never holds, return the exact top-k
    over all pairs (the algorithm's final fallback).

    ``all_k`` uses delta / k (Lemma topkdip).  A has shape (D, L, K, w),
    U (D, L, K).  Returns a dict with the motifs [(dist_d, a, b, dims,
    dist_max)], the stopping (i, j) (None when the exact fallback ran), the
    number of distance computations (verified pairs, repeats included, as
    the paper counts them), the failure bound at return and the number of
    distinct verified pairs."""
    T = np.asarray(T, dtype=np.float64)
    D, n = T.shape
    L, K = A.shape[1], A.shape[2]
    eps = exclusion_zone(w, excl)
    dlt = delta / k if all_k else delta
    keys, _ = hash_all(T, w, A, U, r)
    Z = [znorm_windows(T[f], w) for f in range(D)]
    top, stop, n_dist, pool = momenti_traverse(
        keys, lambda a, b: _pair_distances(Z, a, b), d, k, dlt, r, eps, K)
    if stop is not None:
        i, j = stop
        return {"motifs": top, "stop": stop, "n_dist": n_dist,
                "fail_bound": failure_bound(top[-1][4], i, j, K, L, d, r), "pool": pool}
    return {"motifs": exact_topk_auto(T, w, d, k, excl, fallback_tau), "stop": None,
            "n_dist": n_dist, "fail_bound": 0.0, "pool": pool}


def momenti_multi(T: np.ndarray, w: int, d_low: int, d_high: int, k: int, delta: float,
                  A: np.ndarray, U: np.ndarray, r: float, excl: int | None = None,
                  keys: np.ndarray | None = None):
    """Section 6.3, motifs of every dimensionality d in [d_low, d_high] in
    one traversal: one TOP per d; a verified pair's per-dimension distances
    give dist_d for every d at once, and the pair is offered to the TOP of
    every d not yet confirmed; the collision condition W >= d uses the
    smallest unconfirmed d, which rises as dimensionalities are confirmed;
    after each repetition every unconfirmed d whose TOP is full and passes
    STOP (Algorithm 2 with that d) is confirmed with its own (i, j).  When
    the loop ends, each d still unconfirmed gets the exact top-k (the final
    fallback of Algorithm 1).

    ``keys`` (uint64 (L, M, D)), when given, replaces the keys hashed from
    A, U and r (the traversal then runs on those keys).

    Returns {d: {"motifs", "stop", "fail_bound"}} and the number of
    distance computations under the key "n_dist"."""
    T = np.asarray(T, dtype=np.float64)
    D, n = T.shape
    L, K = A.shape[1], A.shape[2]
    if not 1 <= d_low <= d_high <= D:
        raise ValueError("need 1 <= d_low <= d_high <= D")
    eps = exclusion_zone(w, excl)
    if keys is None:
        keys, _ = hash_all(T, w, A, U, r)
    M = keys.shape[1]
    Z = [znorm_windows(T[f], w) for f in range(D)]
    pools = {d: _Pool(k, eps) for d in range(d_low, d_high + 1)}
    done = {}
    n_dist = 0
    for i in range(K, 0, -1):
        for j in range(1, L + 1):
            open_d = [d for d in pools if d not in done]
            if not open_d:
                break
            d_cur = min(open_d)
            codes = [colliding_pairs(keys[j - 1, :, f], i) for f in range(D)]
            allc = np.concatenate(codes) if codes else np.zeros(0, np.int64)
            uniq, W = np.unique(allc, return_counts=True)
            sel = uniq[W >= d_cur]
            a, b = sel // M, sel % M
            nt = (b - a) > eps
            a, b = a[nt], b[nt]
            if a.size:
                dist = _pair_distances(Z, a, b)
                n_dist += int(a.size)
                for d in open_d:
                    dd, _, dmax, order = _select_d_many(dist, d)
                    pools[d].add_many(a, b, dd, order, dmax)
            for d in open_d:
                top = pools[d].top()
                if len(top) == k and stop_condition(top[-1][4], i, j, K, L, d, delta, r):
                    done[d] = {"motifs": top, "stop": (i, j),
                               "fail_bound": failure_bound(top[-1][4], i, j, K, L, d, r)}
        if len(done) == len(pools):
            break
    out = {}
    for d in pools:
        out[d] = done.get(d) or {"motifs": exact_topk_auto(T, w, d, k, excl), "stop": None,
                                 "fail_bound": 0.0}
    out["n_dist"] = n_dist
    return out


def tensored_keys(T: np.ndarray, w: int, Al: np.ndarray, Ul: np.ndarray, Ar: np.ndarray,
                  Ur: np.ndarray, r: float) -> np.ndarray:
    """Tensoring (Section 6.1): m left and m right hash functions of K/2
    values each (Al, Ar of shape (D, m, K/2, w), Ul, Ur (D, m, K/2));
    repetition j' (0-based) interleaves the values of left function
    j' div m and right function j' mod m, a left value first.  Only K m
    projections per window and dimension are evaluated for m^2
    repetitions.  Returns keys uint64 (m^2, M, D) packed like pack_keys."""
    T = np.asarray(T, dtype=np.float64)
    D = T.shape[0]
    m, half = Al.shape[1], Al.shape[2]
    M = T.shape[1] - w + 1
    keys = np.empty((m * m, M, D), dtype=np.uint64)
    for f in range(D):
        hl, _ = hash_values(T, w, Al, Ul, r, f)                 # (M, m, K/2)
        hr, _ = hash_values(T, w, Ar, Ur, r, f)
        for jj in range(m * m):
            lf, rf = divmod(jj, m)
            h = np.empty((M, 2 * half), dtype=np.int16)
            h[:, 0::2] = hl[:, lf, :]
            h[:, 1::2] = hr[:, rf, :]
            keys[jj, :, f] = pack_keys(h)
    return keys


def momenti_tensored(T: np.ndarray, w: int, d: int, k: int, delta: float, Al: np.ndarray,
                     Ul: np.ndarray, Ar: np.ndarray, Ur: np.ndarray, r: float,
                     excl: int | None = None):
    """Algorithm 1 on tensored keys (``tensored_keys``, L = m^2
    repetitions, K = 2 x the values per function) with STOP on the
    re-derived tensoring bound (``tensoring_failure_bound`` of
    p = P(dist_max)^d); the exact top-k when STOP never holds.  Returns
    the same record as ``momenti``."""
    T = np.asarray(T, dtype=np.float64)
    D = T.shape[0]
    m, K = Al.shape[1], 2 * Al.shape[2]
    L = m * m
    eps = exclusion_zone(w, excl)
    keys = tensored_keys(T, w, Al, Ul, Ar, Ur, r)
    Z = [znorm_windows(T[f], w) for f in range(D)]

    def bound(dist_max, i, j):
        return tensoring_failure_bound(collision_probability(dist_max, r) ** d, i, j, K, L)

    top, stop, n_dist, pool = momenti_traverse(
        keys, lambda a, b: _pair_distances(Z, a, b), d, k, delta, r, eps, K, bound=bound)
    if stop is not None:
        i, j = stop
        return {"motifs": top, "stop": stop, "n_dist": n_dist,
                "fail_bound": bound(top[-1][4], i, j), "pool": pool}
    return {"motifs": exact_topk_auto(T, w, d, k, excl), "stop": None,
            "n_dist": n_dist, "fail_bound": 0.0, "pool": pool}
