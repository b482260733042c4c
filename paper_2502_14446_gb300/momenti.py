"""Thin Python binding of the C ABI in ``include/momenti.h`` (ctypes).

Argument marshalling only: every step of the search runs in the CUDA
library ``libmomenti.so``.  The module raises at import if the library is
missing: there is no CPU fallback.  Series may be numpy arrays (host) or
CUDA torch tensors (device pointers are passed through, with the tensor's
current stream).
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libmomenti.so")

OK = 0
ERR_ARG, ERR_MEMORY, ERR_CUDA, ERR_TIMEOUT, ERR_OVERFLOW, ERR_STATE = -1, -2, -3, -4, -5, -6
F32, F64 = 0, 1
PREC_FP32, PREC_F16X2 = 0, 1
FLAG_TILES_ONLY = 1
FLAG_NO_COST_SWITCH = 2
FLAG_TENSORING = 4
DELTA_PER_MOTIF, DELTA_ALL_K = 0, 1
MAX_D, MAX_K = 64, 8
NOALLOC_MAX_KEYS = 262144

# every symbol include/momenti.h declares
EXPORTS = (
    "momenti_default_params", "momenti_create", "momenti_destroy", "momenti_last_error",
    "momenti_set_hash_params", "momenti_hash_all", "momenti_topk", "momenti_topk_exact",
    "momenti_verify", "momenti_get_info", "momenti_get_window_stats", "momenti_get_keys",
    "momenti_get_index", "momenti_collide", "momenti_launch_count", "momenti_time_kernel",
    "momenti_kernel_time", "momenti_index_sort_noalloc", "momenti_topk_batch",
    "momenti_collision_probability", "momenti_failure_bound", "momenti_top_select",
    "momenti_tensoring_failure_bound", "momenti_get_hash_draws", "momenti_topk_multi",
    "momenti_search_begin", "momenti_search_step", "momenti_search_current",
    "momenti_search_finish",
)


class momenti_params(C.Structure):
    _fields_ = [("w", C.c_int32), ("d", C.c_int32), ("k", C.c_int32), ("delta", C.c_double),
                ("mem_limit", C.c_uint64), ("K", C.c_int32), ("L", C.c_int32), ("r", C.c_double),
                ("excl", C.c_int32), ("seed", C.c_uint64), ("precision", C.c_int32),
                ("delta_mode", C.c_int32), ("flags", C.c_uint32), ("reserved", C.c_uint32)]


class momenti_motif(C.Structure):
    _fields_ = [("a", C.c_int64), ("b", C.c_int64), ("dist_d", C.c_double),
                ("dist_max", C.c_double), ("fail_bound", C.c_double), ("dims_mask", C.c_uint64)]


class momenti_stats(C.Structure):
    _fields_ = [("stop_i", C.c_int32), ("stop_j", C.c_int32), ("K", C.c_int32), ("L", C.c_int32),
                ("r", C.c_double), ("n_windows", C.c_int64), ("n_candidates", C.c_int64),
                ("n_verified", C.c_int64), ("n_pool", C.c_int64), ("fallback", C.c_int32),
                ("n_chunks", C.c_int32), ("t_hash_ms", C.c_double), ("t_sort_ms", C.c_double),
                ("t_traverse_ms", C.c_double), ("t_fallback_ms", C.c_double),
                ("max_rel_err_fp32", C.c_double), ("device_bytes", C.c_uint64),
                ("precision_used", C.c_int32), ("reserved", C.c_int32),
                ("n_rehashed", C.c_uint64), ("n_lb_pruned", C.c_int64), ("t_host_ms", C.c_double),
                ("switch_level", C.c_int32), ("reserved2", C.c_int32),
                ("n_pair_checks", C.c_int64), ("predicted_rest_ms", C.c_double),
                ("predicted_exact_ms", C.c_double)]


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing: build it with "
                          "paper_2502_14446_gb300.build_ext.build() (nvcc, sm_103a)")
    lib = C.CDLL(LIB_PATH)
    P = C.POINTER
    vp = C.c_void_p
    sig = {
        "momenti_default_params": (C.c_int, [P(momenti_params)]),
        "momenti_create": (C.c_int, [P(vp), P(momenti_params)]),
        "momenti_destroy": (None, [vp]),
        "momenti_last_error": (C.c_char_p, [vp]),
        "momenti_set_hash_params": (C.c_int, [vp, C.c_int32, C.c_int32, C.c_int32, C.c_int32,
                                              vp, vp]),
        "momenti_hash_all": (C.c_int, [vp, vp, C.c_int32, C.c_int64, C.c_int32, C.c_int64,
                                       C.c_int32, vp]),
        "momenti_topk": (C.c_int, [vp, P(momenti_motif), P(C.c_int32), P(momenti_stats)]),
        "momenti_topk_exact": (C.c_int, [vp, P(momenti_motif), P(C.c_int32)]),
        "momenti_topk_multi": (C.c_int, [vp, C.c_int32, C.c_int32, P(momenti_motif),
                                         P(C.c_int32), P(C.c_int32), P(momenti_stats)]),
        "momenti_search_begin": (C.c_int, [vp, C.c_int32, C.c_int32]),
        "momenti_search_step": (C.c_int, [vp, C.c_int64, P(C.c_int32)]),
        "momenti_search_current": (C.c_int, [vp, P(momenti_motif), P(C.c_int32), P(C.c_int32)]),
        "momenti_search_finish": (C.c_int, [vp, P(momenti_motif), P(C.c_int32), P(C.c_int32),
                                            P(momenti_stats)]),
        "momenti_verify": (C.c_int, [vp, vp, C.c_int64, vp, vp, vp, C.c_int32]),
        "momenti_get_info": (C.c_int, [vp, P(C.c_int64), P(C.c_int32), P(C.c_int32),
                                       P(C.c_int32), P(C.c_double)]),
        "momenti_get_window_stats": (C.c_int, [vp, vp, vp]),
        "momenti_get_keys": (C.c_int, [vp, C.c_int32, vp]),
        "momenti_get_index": (C.c_int, [vp, C.c_int32, C.c_int32, vp, vp]),
        "momenti_get_hash_draws": (C.c_int, [vp, vp, vp]),
        "momenti_collide": (C.c_int, [vp, C.c_int32, C.c_int32, vp, C.c_int64, P(C.c_int64)]),
        "momenti_launch_count": (C.c_uint64, []),
        "momenti_time_kernel": (C.c_int, [C.c_char_p]),
        "momenti_kernel_time": (C.c_int, [P(C.c_double), P(C.c_uint64)]),
        "momenti_index_sort_noalloc": (C.c_int, [vp, C.c_int64, C.c_int32, vp, vp, vp]),
        "momenti_collision_probability": (C.c_double, [C.c_double, C.c_double]),
        "momenti_failure_bound": (C.c_double, [C.c_double, C.c_int32, C.c_int32, C.c_int32,
                                               C.c_int32, C.c_int32, C.c_double]),
        "momenti_top_select": (C.c_int, [vp, vp, vp, C.c_int64, C.c_int32, C.c_int64,
                                         C.c_int64, vp, P(C.c_int32)]),
        "momenti_tensoring_failure_bound": (C.c_double, [C.c_double, C.c_int32, C.c_int32,
                                                         C.c_int32, C.c_int32]),
        "momenti_topk_batch": (C.c_int, [C.c_int32, P(momenti_params), P(vp), P(C.c_int32),
                                         P(C.c_int64), P(C.c_int32), C.c_int32, C.c_int32,
                                         P(momenti_motif), C.c_int32, P(C.c_int32),
                                         P(momenti_stats), P(C.c_int32), C.c_char_p, C.c_int32]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    return lib


lib = _load()


class MomentiError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"momenti error {code}: {msg}")
        self.code = code


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p)


def default_params(**kw) -> momenti_params:
    p = momenti_params()
    lib.momenti_default_params(C.byref(p))
    for k, v in kw.items():
        setattr(p, k, v)
    return p


def launch_count() -> int:
    """Kernels launched by the library in this process."""
    return int(lib.momenti_launch_count())


def time_kernel(name: str | None):
    """Time every launch of one kernel (CUDA events on its stream)."""
    lib.momenti_time_kernel(name.encode() if name else None)


def kernel_time():
    """(total ms, launches) of the timed kernel since time_kernel()."""
    ms, n = C.c_double(), C.c_uint64()
    rc = lib.momenti_kernel_time(C.byref(ms), C.byref(n))
    if rc != OK:
        raise MomentiError(rc, "momenti_kernel_time")
    return ms.value, int(n.value)


def collision_probability(R: float, r: float) -> float:
    """Eq. (eucl-collision-probability) as the library's search evaluates it."""
    return float(lib.momenti_collision_probability(R, r))


def failure_bound(dist_max: float, i: int, j: int, K: int, L: int, d: int, r: float) -> float:
    """The bound of Lemma stop that Algorithm 2 compares with delta (i, j 1-based)."""
    return float(lib.momenti_failure_bound(dist_max, i, j, K, L, d, r))


def tensoring_failure_bound(p: float, i: int, j: int, K: int, L: int) -> float:
    """The re-derived miss bound of tensoring (L a square, K even)."""
    return float(lib.momenti_tensoring_failure_bound(p, i, j, K, L))


def top_select(dd, a, b, k: int, eps: int, batch: int = 1 << 30):
    """TOP over given candidate pairs through the search's pool, fed
    ``batch`` pairs at a time; returns the positions of TOP's pairs."""
    dd = np.ascontiguousarray(dd, dtype=np.float32)
    a = np.ascontiguousarray(a, dtype=np.int64)
    b = np.ascontiguousarray(b, dtype=np.int64)
    if not (dd.shape == a.shape == b.shape and dd.ndim == 1):
        raise ValueError("dd, a, b: equal-length vectors")
    idx = np.zeros(max(k, 1), dtype=np.int64)
    n = C.c_int32()
    rc = lib.momenti_top_select(_ptr(dd), _ptr(a), _ptr(b), dd.size, k, eps, batch, _ptr(idx),
                                C.byref(n))
    if rc != OK:
        raise MomentiError(rc, "momenti_top_select")
    return [int(q) for q in idx[:n.value]]


def topk_batch(params, series_list, threads: int = 8):
    """momenti_topk_batch: search every series of ``series_list`` ((D, n)
    host arrays, or CUDA tensors all on the device) with ``params[b]`` (a
    list of momenti_params or of keyword dicts for default_params).
    Returns ``[(motifs, stats)]`` as Momenti.topk gives them, in order.
    Raises MomentiError (naming the first failing series) if any failed."""
    B = len(series_list)
    assert len(params) == B
    P = (momenti_params * B)()
    for b, p in enumerate(params):
        P[b] = p if isinstance(p, momenti_params) else default_params(**p)
    keep = []
    on_dev = int(bool(B) and hasattr(series_list[0], "is_cuda") and series_list[0].is_cuda)
    ptrs = (C.c_void_p * B)()
    dt = (C.c_int32 * B)()
    ns = (C.c_int64 * B)()
    Ds = (C.c_int32 * B)()
    for b, x in enumerate(series_list):
        if on_dev:
            import torch
            assert x.is_cuda and x.dim() == 2 and x.is_contiguous()
            ptrs[b] = x.data_ptr()
            dt[b] = F64 if x.dtype == torch.float64 else F32
        else:
            x = np.ascontiguousarray(np.asarray(x))
            if x.dtype not in (np.float32, np.float64):
                x = x.astype(np.float64)
            ptrs[b] = x.ctypes.data
            dt[b] = F64 if x.dtype == np.float64 else F32
        Ds[b], ns[b] = x.shape
        keep.append(x)
    kmax = max([P[b].k for b in range(B)] + [1])
    out = (momenti_motif * (B * kmax))()
    n_out = (C.c_int32 * B)()
    st = (momenti_stats * B)()
    rcs = (C.c_int32 * B)()
    err = C.create_string_buffer(512)
    rc = lib.momenti_topk_batch(B, P, ptrs, dt, ns, Ds, on_dev, threads, out, kmax, n_out, st,
                                rcs, err, 512)
    if rc != OK:
        raise MomentiError(rc, f"momenti_topk_batch: {err.value.decode() or 'invalid arguments'}")
    res = []
    for b in range(B):
        motifs = Momenti._motifs(out[b * kmax:(b + 1) * kmax], n_out[b])
        res.append((motifs, {name: getattr(st[b], name) for name, _ in momenti_stats._fields_}))
    return res


class Momenti:
    """One search handle: ``hash_all`` builds the index, ``topk`` searches."""

    def __init__(self, params: momenti_params | None = None, **kw):
        self.params = params if params is not None else default_params(**kw)
        if params is not None:
            for k, v in kw.items():
                setattr(self.params, k, v)
        h = C.c_void_p()
        rc = lib.momenti_create(C.byref(h), C.byref(self.params))
        if rc != OK:
            raise MomentiError(rc, "momenti_create: invalid parameters")
        self.h = h
        self._keep = None

    def close(self):
        if self.h:
            lib.momenti_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def _check(self, rc, what):
        if rc != OK:
            msg = lib.momenti_last_error(self.h)
            raise MomentiError(rc, f"{what}: {msg.decode() if msg else ''}")

    def set_hash_params(self, A: np.ndarray, U: np.ndarray):
        A = np.ascontiguousarray(A, dtype=np.float32)
        U = np.ascontiguousarray(U, dtype=np.float32)
        D, L, K, w = A.shape
        assert U.shape == (D, L, K)
        self._check(lib.momenti_set_hash_params(self.h, D, L, K, w, _ptr(A), _ptr(U)),
                    "momenti_set_hash_params")

    def hash_all(self, series, stream=None):
        """series: (D, n) numpy array (host) or CUDA torch tensor (device)."""
        if hasattr(series, "is_cuda") and series.is_cuda:
            import torch
            assert series.dim() == 2 and series.stride(1) == 1
            dtype = F64 if series.dtype == torch.float64 else F32
            assert series.dtype in (torch.float32, torch.float64)
            D, n = series.shape
            if stream is None:
                stream = torch.cuda.current_stream(series.device).cuda_stream
            self._keep = series
            rc = lib.momenti_hash_all(self.h, C.c_void_p(series.data_ptr()), dtype, n, D,
                                      series.stride(0), 1, C.c_void_p(stream))
        else:
            arr = np.asarray(series)
            if arr.dtype not in (np.float32, np.float64):
                arr = arr.astype(np.float64)
            arr = np.ascontiguousarray(arr)
            D, n = arr.shape
            dtype = F64 if arr.dtype == np.float64 else F32
            rc = lib.momenti_hash_all(self.h, _ptr(arr), dtype, n, D, n, 0,
                                      C.c_void_p(stream or 0))
        self._check(rc, "momenti_hash_all")

    def info(self):
        M, D, L, K, r = C.c_int64(), C.c_int32(), C.c_int32(), C.c_int32(), C.c_double()
        self._check(lib.momenti_get_info(self.h, C.byref(M), C.byref(D), C.byref(L), C.byref(K),
                                         C.byref(r)), "momenti_get_info")
        return {"M": M.value, "D": D.value, "L": L.value, "K": K.value, "r": r.value}

    @staticmethod
    def _motifs(buf, n):
        out = []
        for q in range(n):
            m = buf[q]
            dims = tuple(f for f in range(64) if m.dims_mask >> f & 1)
            out.append({"a": m.a, "b": m.b, "dist_d": m.dist_d, "dist_max": m.dist_max,
                        "fail_bound": m.fail_bound, "dims": dims})
        return out

    def topk(self):
        k = self.params.k
        buf = (momenti_motif * k)()
        n = C.c_int32()
        st = momenti_stats()
        self._check(lib.momenti_topk(self.h, buf, C.byref(n), C.byref(st)), "momenti_topk")
        stats = {name: getattr(st, name) for name, _ in momenti_stats._fields_}
        return self._motifs(buf, n.value), stats

    def topk_multi(self, d_low: int, d_high: int):
        """Section 6.3: {d: (motifs, (stop_i, stop_j))} for d_low..d_high,
        and the stats of the traversal."""
        k = self.params.k
        nd = d_high - d_low + 1
        buf = (momenti_motif * (k * max(nd, 1)))()
        n = (C.c_int32 * max(nd, 1))()
        stops = (C.c_int32 * (2 * max(nd, 1)))()
        st = momenti_stats()
        self._check(lib.momenti_topk_multi(self.h, d_low, d_high, buf, n, stops, C.byref(st)),
                    "momenti_topk_multi")
        out = {}
        for q in range(nd):
            out[d_low + q] = (self._motifs(buf[q * k:(q + 1) * k], n[q]),
                              (stops[2 * q], stops[2 * q + 1]))
        return out, {name: getattr(st, name) for name, _ in momenti_stats._fields_}

    # ---- anytime search ----
    def search_begin(self, d_low: int | None = None, d_high: int | None = None):
        d_low = self.params.d if d_low is None else d_low
        d_high = d_low if d_high is None else d_high
        self._search = (d_low, d_high)
        self._check(lib.momenti_search_begin(self.h, d_low, d_high), "momenti_search_begin")

    def search_step(self, max_reps: int = 1) -> bool:
        """Advances the search; True once the traversal has ended."""
        ended = C.c_int32()
        self._check(lib.momenti_search_step(self.h, max_reps, C.byref(ended)), "momenti_search_step")
        return bool(ended.value)

    def search_current(self):
        """({d: motifs with their current miss bounds}, (i, j, ended))."""
        d_low, d_high = self._search
        k, nd = self.params.k, d_high - d_low + 1
        buf = (momenti_motif * (k * nd))()
        n = (C.c_int32 * nd)()
        cur = (C.c_int32 * 3)()
        self._check(lib.momenti_search_current(self.h, buf, n, cur), "momenti_search_current")
        return ({d_low + q: self._motifs(buf[q * k:(q + 1) * k], n[q]) for q in range(nd)},
                (cur[0], cur[1], bool(cur[2])))

    def search_finish(self):
        """The final results, as topk_multi returns them."""
        d_low, d_high = self._search
        k, nd = self.params.k, d_high - d_low + 1
        buf = (momenti_motif * (k * nd))()
        n = (C.c_int32 * nd)()
        stops = (C.c_int32 * (2 * nd))()
        st = momenti_stats()
        self._check(lib.momenti_search_finish(self.h, buf, n, stops, C.byref(st)),
                    "momenti_search_finish")
        out = {d_low + q: (self._motifs(buf[q * k:(q + 1) * k], n[q]),
                           (stops[2 * q], stops[2 * q + 1])) for q in range(nd)}
        return out, {name: getattr(st, name) for name, _ in momenti_stats._fields_}

    def topk_exact(self):
        k = self.params.k
        buf = (momenti_motif * k)()
        n = C.c_int32()
        self._check(lib.momenti_topk_exact(self.h, buf, C.byref(n)), "momenti_topk_exact")
        return self._motifs(buf, n.value)

    def verify(self, pairs, fp64: bool = False):
        pairs = np.ascontiguousarray(np.asarray(pairs, dtype=np.int64).reshape(-1, 2))
        m = pairs.shape[0]
        D = self.info()["D"]
        per = np.zeros((m, D))
        dd = np.zeros(m)
        mask = np.zeros(m, dtype=np.uint64)
        self._check(lib.momenti_verify(self.h, _ptr(pairs), m, _ptr(per), _ptr(dd), _ptr(mask),
                                       1 if fp64 else 0), "momenti_verify")
        return per, dd, mask

    def window_stats(self):
        inf = self.info()
        mu = np.zeros((inf["D"], inf["M"]))
        sd = np.zeros((inf["D"], inf["M"]))
        self._check(lib.momenti_get_window_stats(self.h, _ptr(mu), _ptr(sd)),
                    "momenti_get_window_stats")
        return mu, sd

    def keys(self, j: int) -> np.ndarray:
        inf = self.info()
        out = np.zeros((inf["M"], inf["D"]), dtype=np.uint64)
        self._check(lib.momenti_get_keys(self.h, j, _ptr(out)), "momenti_get_keys")
        return out

    def hash_draws(self):
        """(a (D, L, K, w), u (D, L, K)) float32: the hash functions' random
        numbers of the current index (under tensoring the 2m half functions
        of K/2 values: a (D, 2m, K/2, w))."""
        inf = self.info()
        nf, kf = inf["L"], inf["K"]
        if self.params.flags & FLAG_TENSORING:            # 2m half functions of K/2 values
            nf, kf = 2 * int(round(inf["L"] ** 0.5)), inf["K"] // 2
        a = np.zeros((inf["D"], nf, kf, self.params.w), dtype=np.float32)
        u = np.zeros((inf["D"], nf, kf), dtype=np.float32)
        self._check(lib.momenti_get_hash_draws(self.h, _ptr(a), _ptr(u)), "momenti_get_hash_draws")
        return a, u

    def index(self, j: int, f: int):
        M = self.info()["M"]
        order = np.zeros(M, dtype=np.uint32)
        lcp = np.zeros(M, dtype=np.uint8)
        self._check(lib.momenti_get_index(self.h, j, f, _ptr(order), _ptr(lcp)),
                    "momenti_get_index")
        return order, lcp

    def collide(self, i: int, j: int, cap: int = 1 << 22) -> np.ndarray:
        out = np.zeros((cap, 2), dtype=np.int64)
        cnt = C.c_int64()
        self._check(lib.momenti_collide(self.h, i, j, _ptr(out), cap, C.byref(cnt)),
                    "momenti_collide")
        if cnt.value > cap:
            return self.collide(i, j, int(cnt.value))
        return out[:cnt.value]
