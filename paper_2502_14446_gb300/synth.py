"""Seeded synthetic inputs for the motif search, shared by the tests, the
benchmark and the CPU oracle.

This module holds no arithmetic of the method itself: it only draws random
numbers.  It produces

* multidimensional series that stand in for the paper's real sensor datasets
  (Section 7, Table 1: random walks, sinusoids, sparse spikes, Gaussian noise)
  with motifs planted in a chosen subset of dimensions (Definition of the
  d-dimensional motif, Section 3.1);
* the random numbers the hash family of Eq. (drp) draws: the projection
  vectors ``a ~ N(0, 1)^w`` and the offsets ``b ~ U[0, r]``, the latter as a
  fraction ``u ~ U[0, 1)`` so that ``b = u * r`` once ``r`` is known.

Projection vectors are rounded to the nearest IEEE half-precision value, so
that the same numbers can be fed unchanged to a half-precision tensor-core
product and to a float64 CPU computation.

All draws use numpy's counter-based Philox generator, keyed by the seed.
"""
from __future__ import annotations

from dataclasses import dataclass, field
import math

import numpy as np


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.Philox(int(seed)))


@dataclass
class Workload:
    """A synthetic problem instance: the series plus the search parameters."""
    name: str
    series: np.ndarray            # shape (D, n), float32 or float64, C-contiguous
    w: int
    d: int
    k: int
    delta: float
    mem_limit: int = 0            # bytes, 0 = library default
    planted: list = field(default_factory=list)   # [(a, b, dims)] planted motif pairs
    seed: int = 0

    @property
    def D(self) -> int:
        return int(self.series.shape[0])

    @property
    def n(self) -> int:
        return int(self.series.shape[1])


# --------------------------------------------------------------------------
# series components
# --------------------------------------------------------------------------

def random_walk(rng: np.random.Generator, D: int, n: int, step: float = 1.0) -> np.ndarray:
    """Gaussian random walk per dimension, unit steps by default."""
    return np.cumsum(rng.standard_normal((D, n)) * step, axis=1)


def sinusoids(rng: np.random.Generator, D: int, n: int, count: int = 3,
              period=(50.0, 2000.0), amplitude=(1.0, 5.0)) -> np.ndarray:
    """Sum of ``count`` sinusoids per dimension with random period, amplitude
    and phase."""
    t = np.arange(n, dtype=np.float64)
    out = np.zeros((D, n))
    for f in range(D):
        for _ in range(count):
            p = rng.uniform(*period)
            amp = rng.uniform(*amplitude)
            ph = rng.uniform(0.0, 2.0 * math.pi)
            out[f] += amp * np.sin(2.0 * math.pi * t / p + ph)
    return out


def spikes(rng: np.random.Generator, D: int, n: int, rate: float, amplitude: float) -> np.ndarray:
    """Sparse Bernoulli(rate) spikes of +-amplitude."""
    mask = rng.random((D, n)) < rate
    sign = np.where(rng.random((D, n)) < 0.5, -1.0, 1.0)
    return mask * sign * amplitude


def _pick_offsets(rng: np.random.Generator, count: int, n: int, w: int, gap: int) -> list[int]:
    """``count`` window offsets in [0, n-w], pairwise at least ``gap`` apart."""
    M = n - w + 1
    for _ in range(10000):
        offs = sorted(int(x) for x in rng.integers(0, M, size=count))
        if all(offs[i + 1] - offs[i] >= gap for i in range(count - 1)):
            return offs
    # crowded: draw in the range left after reserving the gaps, then spread
    free = M - (count - 1) * gap
    if free <= 0:
        raise ValueError("cannot place planted motifs: series too short")
    base = sorted(int(x) for x in rng.integers(0, free, size=count))
    return [b + i * gap for i, b in enumerate(base)]


def plant_motifs(rng: np.random.Generator, T: np.ndarray, w: int, n_motifs: int,
                 dims_per_motif: int, noise: float, fixed_dims=None) -> list:
    """Plant ``n_motifs`` pairs of similar windows into ``T`` (in place).

    Each motif is one shape (a standardised random-walk segment of length w)
    written at two offsets.  In each chosen dimension the shape replaces the
    host window, keeping the host window's level and spread, and gets
    independent Gaussian noise of ``noise`` times that spread.  All planted
    windows are at least 2w apart.  Returns ``[(a, b, dims)]``.
    """
    D, n = T.shape
    offs = _pick_offsets(rng, 2 * n_motifs, n, w, 2 * w)
    order = rng.permutation(len(offs))
    out = []
    for m in range(n_motifs):
        a, b = sorted((offs[order[2 * m]], offs[order[2 * m + 1]]))
        if fixed_dims is not None:
            dims = sorted(fixed_dims)
        else:
            dims = sorted(int(x) for x in rng.choice(D, size=dims_per_motif, replace=False))
        shape = np.cumsum(rng.standard_normal(w))
        shape = (shape - shape.mean()) / shape.std()
        for f in dims:
            for off in (a, b):
                host = T[f, off:off + w]
                lvl, spread = host.mean(), host.std()
                if spread <= 0:
                    spread = 1.0
                T[f, off:off + w] = lvl + spread * (shape + noise * rng.standard_normal(w))
        out.append((a, b, dims))
    return out


# --------------------------------------------------------------------------
# the workloads
# --------------------------------------------------------------------------

def plain_small(seed: int = 0, n: int = 5000, D: int = 4) -> Workload:
    """Plain method, single series: D=4, n=5000, w=100, d=2, k=5, delta=0.1,
    float64 Gaussian random walks with two motifs planted in dims {0, 2}."""
    rng = _rng(seed)
    T = random_walk(rng, D, n)
    planted = plant_motifs(rng, T, 100, 2, 2, 0.05, fixed_dims=(0, 2))
    return Workload("plain_small", np.ascontiguousarray(T, dtype=np.float64), 100, 2, 5, 0.1,
                    planted=planted, seed=seed)


def plain_fp32(seed: int = 0, n: int = 100_000, D: int = 8, w: int = 300) -> Workload:
    """Plain method, float32: D=8, n=100000, w=300, d=3, k=10, delta=0.05.
    Random walk + 3 sinusoids (period U[50, 2000]) + N(0, 0.1) noise, five
    motifs planted in 3 random dims each; memory limit 8 GB."""
    rng = _rng(1000 + seed)
    T = random_walk(rng, D, n) + sinusoids(rng, D, n) + 0.1 * rng.standard_normal((D, n))
    planted = plant_motifs(rng, T, w, 5, 3, 0.05)
    return Workload("plain_fp32", np.ascontiguousarray(T, dtype=np.float32), w, 3, 10, 0.05,
                    mem_limit=8 << 30, planted=planted, seed=seed)


def precision_form(seed: int = 0, n: int = 1_000_000, D: int = 32, w: int = 500) -> Workload:
    """Precision form: D=32, n=1e6, w=500, d=8, k=10, delta=0.01, float32.
    Random walk + sinusoids + Bernoulli(1e-4) spikes of 5 step-sigmas, ten
    motifs planted in 8 dims each."""
    rng = _rng(2000 + seed)
    T = (random_walk(rng, D, n) + sinusoids(rng, D, n)
         + spikes(rng, D, n, 1e-4, 5.0) + 0.1 * rng.standard_normal((D, n)))
    planted = plant_motifs(rng, T, w, 10, 8, 0.05)
    return Workload("precision_form", np.ascontiguousarray(T, dtype=np.float32), w, 8, 10, 0.01,
                    planted=planted, seed=seed)


def batch_form(seed: int = 0, count: int = 256, n_lo: int = 2000, n_hi: int = 200_000) -> list:
    """Batching form: ``count`` independent float32 series with log-uniform
    n in [n_lo, n_hi], D uniform in [3, 16], w in {50, 100, 200},
    d = ceil(D/3), k=5, delta=0.05; random walk + noise with 2 planted
    motifs each."""
    rng = _rng(3000 + seed)
    out = []
    for s in range(count):
        n = int(round(math.exp(rng.uniform(math.log(n_lo), math.log(n_hi)))))
        D = int(rng.integers(3, 17))
        w = int(rng.choice([50, 100, 200]))
        n = max(n, 8 * w + 16)
        d = int(math.ceil(D / 3))
        T = random_walk(rng, D, n) + 0.1 * rng.standard_normal((D, n))
        planted = plant_motifs(rng, T, w, 2, d, 0.05)
        out.append(Workload(f"batch_{s}", np.ascontiguousarray(T, dtype=np.float32), w, d, 5, 0.05,
                            planted=planted, seed=seed))
    return out


def large_form(seed: int = 0, n: int = 10_000_000, D: int = 64, w: int = 1000) -> Workload:
    """Large memory-bounded form: D=64, n=1e7, w=1000, d=16, k=10,
    delta=0.01, float32, 64 GB limit; 20 motifs planted in 16 dims each."""
    rng = _rng(4000 + seed)
    T = random_walk(rng, D, n) + sinusoids(rng, D, n) + 0.1 * rng.standard_normal((D, n))
    planted = plant_motifs(rng, T, w, 20, 16, 0.05)
    return Workload("large_form", np.ascontiguousarray(T, dtype=np.float32), w, 16, 10, 0.01,
                    mem_limit=64 << 30, planted=planted, seed=seed)


def tiny(seed: int, n: int, D: int, w: int, d: int, k: int = 2, n_motifs: int = 1,
         dtype=np.float64, noise: float = 0.05) -> Workload:
    """Small random-walk instance for brute-force cross checks."""
    rng = _rng(5000 + seed)
    T = random_walk(rng, D, n)
    planted = []
    if n_motifs:
        planted = plant_motifs(rng, T, w, n_motifs, d, noise)
    return Workload(f"tiny_{seed}", np.ascontiguousarray(T, dtype=dtype), w, d, k, 0.1,
                    planted=planted, seed=seed)


def scalability(seed: int = 0, n: int = 100_000, noise: float = 0.1) -> Workload:
    """The synthetic scalability workload of Section 7: D=5 Gaussian random
    walks of length n, one sinusoidal motif of length w=300 planted in dims
    {0, 1} at two offsets 2w or more apart (one period of a sine, written
    with the host window's level and spread), perturbed by Gaussian noise of
    ``noise`` times that spread (a low-contrast motif); d=2, k=1,
    delta=0.05."""
    rng = _rng(6000 + seed)
    D, w = 5, 300
    T = random_walk(rng, D, n)
    a, b = sorted(_pick_offsets(rng, 2, n, w, 2 * w))
    shape = np.sin(2 * np.pi * np.arange(w) / w)
    shape = (shape - shape.mean()) / shape.std()
    for f in (0, 1):
        for off in (a, b):
            host = T[f, off:off + w]
            lvl, spread = host.mean(), host.std()
            T[f, off:off + w] = lvl + (spread if spread > 0 else 1.0) * (
                shape + noise * rng.standard_normal(w))
    return Workload("scalability", np.ascontiguousarray(T, dtype=np.float32), w, 2, 1, 0.05,
                    planted=[(a, b, [0, 1])], seed=seed)


def with_noise_dims(wl: Workload, extra: int, seed: int = 0) -> Workload:
    """The robustness workload of Section 7 (impact of noise): ``wl`` with
    ``extra`` more dimensions appended, each an independent Gaussian random
    walk that holds no planted motif."""
    rng = _rng(9000 + seed)
    noise = random_walk(rng, extra, wl.n).astype(wl.series.dtype)
    T = np.ascontiguousarray(np.concatenate([wl.series, noise], axis=0))
    return Workload(f"{wl.name}+{extra}noise", T, wl.w, wl.d, wl.k, wl.delta, wl.mem_limit,
                    planted=list(wl.planted), seed=wl.seed)


# --------------------------------------------------------------------------
# random numbers of the hash family, Eq. (drp)
# --------------------------------------------------------------------------

def hash_draws(D: int, L: int, K: int, w: int, seed: int = 0):
    """Draw the projection vectors and offset fractions of D*L*K hash
    functions.

    Returns ``(A, U)``: ``A`` float32 of shape (D, L, K, w) with N(0, 1)
    entries rounded to half precision, ``U`` float32 of shape (D, L, K) with
    U[0, 1) entries (the offset is ``b = U * r``).
    """
    rng = _rng(7000 + seed)
    A = rng.standard_normal((D, L, K, w)).astype(np.float16).astype(np.float32)
    U = rng.random((D, L, K)).astype(np.float32)
    U = np.minimum(U, np.float32(1.0) - np.float32(2.0 ** -24))
    return np.ascontiguousarray(A), np.ascontiguousarray(U)
