// Device code of candidate verification and of the exact all-pairs path
// (the kernels, their device helpers, shared-memory sizes and launch
// templates).  Included by k_verify.cu and by the translation units that
// instantiate the 64-dimension sweeps (k_wide64_*.cu), so that the heavy
// instantiations compile in parallel; every definition has internal
// linkage.  What the kernels compute is stated in k_verify.cu's header.
#pragma once

#include "internal.h"

#include <algorithm>
#include <cstdint>

namespace momenti {

namespace {

__device__ __forceinline__ float warp_sum(float v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ double warp_sum(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
template <typename T>
__device__ __forceinline__ T warp_max(T v) {
  for (int o = 16; o > 0; o >>= 1) v = max(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

struct VerifyOut {
  double dist_d, dist_max;
  uint64_t mask;
};

// Distances of one pair; lane f (and f - 32) ends up holding dimension f.
template <typename T>
__device__ void pair_distances(const Index& ix, uint32_t a, uint32_t b, T dist[2]) {
  const int lane = threadIdx.x & 31;
  dist[0] = dist[1] = T(0);
  for (int f = 0; f < ix.D; ++f) {
    const int64_t oa = int64_t(f) * ix.M + a, ob = int64_t(f) * ix.M + b;
    const float* xa = ix.xs_hi + int64_t(f) * ix.n + a;
    const float* xb = ix.xs_hi + int64_t(f) * ix.n + b;
    const float* la = ix.has_lo ? ix.xs_lo + int64_t(f) * ix.n + a : nullptr;
    const float* lb = ix.has_lo ? ix.xs_lo + int64_t(f) * ix.n + b : nullptr;
    T s = T(0);
    if constexpr (sizeof(T) == 4) {
      const float m0a = ix.mu_hi[oa], m1a = ix.mu_lo[oa], isa = ix.inv_sig[oa];
      const float m0b = ix.mu_hi[ob], m1b = ix.mu_lo[ob], isb = ix.inv_sig[ob];
      for (int t = lane; t < ix.w; t += 32) {
        float za = ((xa[t] - m0a) + ((la ? la[t] : 0.f) - m1a)) * isa;
        float zb = ((xb[t] - m0b) + ((lb ? lb[t] : 0.f) - m1b)) * isb;
        float dd = za - zb;
        s = fmaf(dd, dd, s);
      }
    } else {
      const double ma = ix.mu[oa], mb = ix.mu[ob];
      const double sa = ix.sig[oa], sb = ix.sig[ob];
      const bool fa = sa <= kFlatRel * (1.0 + fabs(ma)), fb = sb <= kFlatRel * (1.0 + fabs(mb));
      const double isa = fa ? 0.0 : 1.0 / sa, isb = fb ? 0.0 : 1.0 / sb;
      for (int t = lane; t < ix.w; t += 32) {
        double va = double(xa[t]) + (la ? double(la[t]) : 0.0);
        double vb = double(xb[t]) + (lb ? double(lb[t]) : 0.0);
        double dd = (va - ma) * isa - (vb - mb) * isb;
        s = fma(dd, dd, s);
      }
    }
    s = warp_sum(s);
    if (lane == (f & 31)) dist[f >> 5] = sqrt(s);
  }
}

// Sum of the d smallest of D per-lane distances (ties to the lower index).
template <typename T>
__device__ VerifyOut select_d(const T dist[2], int D, int d) {
  const int lane = threadIdx.x & 31;
  int rank[2] = {0, 0};
  for (int g = 0; g < D; ++g) {
    T vg = __shfl_sync(0xffffffffu, dist[g >> 5], g & 31);
    for (int h = 0; h < 2; ++h) {
      int f = lane + 32 * h;
      if (f < D && (vg < dist[h] || (vg == dist[h] && g < f))) ++rank[h];
    }
  }
  T sum = 0, mx = 0;
  bool sel0 = lane < D && rank[0] < d, sel1 = lane + 32 < D && rank[1] < d;
  if (sel0) { sum += dist[0]; mx = dist[0]; }
  if (sel1) { sum += dist[1]; mx = max(mx, dist[1]); }
  sum = warp_sum(sum);
  mx = warp_max(mx);
  uint64_t m0 = __ballot_sync(0xffffffffu, sel0), m1 = __ballot_sync(0xffffffffu, sel1);
  return VerifyOut{double(sum), double(mx), m0 | (m1 << 32)};
}

// Per-dimension distances of one pair in FP32 with all dims' partial sums
// kept per lane (loads of every dim in flight together), then the D warp
// reductions interleaved; lane f (and f - 32) ends with dimension f.
template <int DM>
__device__ __forceinline__ void pair_distances_fast(const Index& ix, uint32_t a, uint32_t b,
                                                    float dist[2]) {
  const int lane = threadIdx.x & 31;
  float acc[DM];
#pragma unroll
  for (int f = 0; f < DM; ++f) acc[f] = 0.f;
#pragma unroll
  for (int f = 0; f < DM; ++f) {
    if (f < ix.D) {
      const int64_t oa = int64_t(f) * ix.M + a, ob = int64_t(f) * ix.M + b;
      const float m0a = ix.mu_hi[oa], m1a = ix.mu_lo[oa], isa = ix.inv_sig[oa];
      const float m0b = ix.mu_hi[ob], m1b = ix.mu_lo[ob], isb = ix.inv_sig[ob];
      const float* xa = ix.xs_hi + int64_t(f) * ix.n + a;
      const float* xb = ix.xs_hi + int64_t(f) * ix.n + b;
      const float* la = ix.has_lo ? ix.xs_lo + int64_t(f) * ix.n + a : nullptr;
      const float* lb = ix.has_lo ? ix.xs_lo + int64_t(f) * ix.n + b : nullptr;
      float s = 0.f;
      for (int t = lane; t < ix.w; t += 32) {
        float za = ((xa[t] - m0a) + ((la ? la[t] : 0.f) - m1a)) * isa;
        float zb = ((xb[t] - m0b) + ((lb ? lb[t] : 0.f) - m1b)) * isb;
        float dd = za - zb;
        s = fmaf(dd, dd, s);
      }
      acc[f] = s;
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1)
#pragma unroll
    for (int f = 0; f < DM; ++f) acc[f] += __shfl_xor_sync(0xffffffffu, acc[f], o);
  dist[0] = dist[1] = 0.f;
#pragma unroll
  for (int f = 0; f < DM; ++f)
    if (f < ix.D && lane == (f & 31)) dist[f >> 5] = sqrtf(acc[f]);
}

template <int DP>
__device__ __forceinline__ void load_row(const float* __restrict__ base, int64_t t, float (&v)[DP]) {
  const float4* p = reinterpret_cast<const float4*>(base + t * DP);
#pragma unroll
  for (int q = 0; q < DP / 4; ++q) {
    const float4 u = p[q];
    v[4 * q] = u.x; v[4 * q + 1] = u.y; v[4 * q + 2] = u.z; v[4 * q + 3] = u.w;
  }
}

// The same through the read-only path with 256-bit loads (DP a multiple of
// 8, rows 32-byte aligned): a lane's row is whole 32-byte sectors, one
// instruction per 8 values.
template <int DP>
__device__ __forceinline__ void load_row_v8(const float* __restrict__ base, int64_t t, float (&v)[DP]) {
  static_assert(DP % 8 == 0, "rows of whole 32-byte sectors");
  const float* p = base + t * DP;
#pragma unroll
  for (int q = 0; q < DP / 8; ++q)
    asm("ld.global.nc.v8.f32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
        : "=f"(v[8 * q]), "=f"(v[8 * q + 1]), "=f"(v[8 * q + 2]), "=f"(v[8 * q + 3]),
          "=f"(v[8 * q + 4]), "=f"(v[8 * q + 5]), "=f"(v[8 * q + 6]), "=f"(v[8 * q + 7])
        : "l"(p + 8 * q));
}

// Column rows of the statistics sweeps: 256-bit loads where a row is whole sectors.
template <int DP>
__device__ __forceinline__ void load_col(const float* __restrict__ base, int64_t t, float (&v)[DP]) {
  if constexpr (DP % 8 == 0) load_row_v8<DP>(base, t, v);
  else load_row<DP>(base, t, v);
}

// dist_d of a pair from per-dim distances (registers), the d smallest.
template <int DM>
__device__ __forceinline__ float sum_d_smallest(const float (&v)[DM], int D, int d) {
  float best[DM];
#pragma unroll
  for (int q = 0; q < DM; ++q) best[q] = INFINITY;
#pragma unroll
  for (int f = 0; f < DM; ++f) {
    if (f < D) {
      float x = v[f];
      // insert x into the sorted prefix best[0..d)
#pragma unroll
      for (int q = DM - 1; q >= 0; --q) {
        if (q < d) {
          float prev = q > 0 ? best[q - 1] : -INFINITY;
          if (x < best[q]) best[q] = x >= prev ? x : prev;
        }
      }
    }
  }
  float s = 0.f;
#pragma unroll
  for (int q = 0; q < DM; ++q)
    if (q < d) s += best[q];
  return s;
}

// Window statistics of window a from the point-major copy: 3 rows of DP.
template <int DP>
__device__ __forceinline__ void load_stats(const Index& ix, uint32_t a, float (&mh)[DP],
                                           float (&ml)[DP], float (&is)[DP]) {
  const float* base = ix.stT + int64_t(a) * 3 * DP;
  load_row<DP>(base, 0, mh);
  load_row<DP>(base + DP, 0, ml);
  load_row<DP>(base + 2 * DP, 0, is);
}

// Point-major form (D <= 8): each lane reads all dims of a time point of
// both windows with float4 loads.  Padding dims have 1/sigma = 0 and add 0.
template <int DP, bool LO>
__device__ __forceinline__ void pair_distances_pm(const Index& ix, uint32_t a, uint32_t b,
                                                  float dist[2]) {
  const int lane = threadIdx.x & 31;
  float m0a[DP], m1a[DP], isa[DP], m0b[DP], m1b[DP], isb[DP], acc[DP];
  load_stats<DP>(ix, a, m0a, m1a, isa);
  load_stats<DP>(ix, b, m0b, m1b, isb);
#pragma unroll
  for (int f = 0; f < DP; ++f) acc[f] = 0.f;
  const float4* pa = reinterpret_cast<const float4*>(ix.xT + int64_t(a) * DP);
  const float4* pb = reinterpret_cast<const float4*>(ix.xT + int64_t(b) * DP);
  const float4* la = LO ? reinterpret_cast<const float4*>(ix.xlT + int64_t(a) * DP) : nullptr;
  const float4* lb = LO ? reinterpret_cast<const float4*>(ix.xlT + int64_t(b) * DP) : nullptr;
  for (int t = lane; t < ix.w; t += 32) {
    float xa[DP], xb[DP], ya[DP], yb[DP];
#pragma unroll
    for (int v = 0; v < DP / 4; ++v) {
      const float4 qa = pa[int64_t(t) * (DP / 4) + v], qb = pb[int64_t(t) * (DP / 4) + v];
      xa[4 * v] = qa.x; xa[4 * v + 1] = qa.y; xa[4 * v + 2] = qa.z; xa[4 * v + 3] = qa.w;
      xb[4 * v] = qb.x; xb[4 * v + 1] = qb.y; xb[4 * v + 2] = qb.z; xb[4 * v + 3] = qb.w;
      if (LO) {
        const float4 ra = la[int64_t(t) * (DP / 4) + v], rb = lb[int64_t(t) * (DP / 4) + v];
        ya[4 * v] = ra.x; ya[4 * v + 1] = ra.y; ya[4 * v + 2] = ra.z; ya[4 * v + 3] = ra.w;
        yb[4 * v] = rb.x; yb[4 * v + 1] = rb.y; yb[4 * v + 2] = rb.z; yb[4 * v + 3] = rb.w;
      }
    }
#pragma unroll
    for (int f = 0; f < DP; ++f) {
      const float za = ((xa[f] - m0a[f]) + ((LO ? ya[f] : 0.f) - m1a[f])) * isa[f];
      const float zb = ((xb[f] - m0b[f]) + ((LO ? yb[f] : 0.f) - m1b[f])) * isb[f];
      const float dd = za - zb;
      acc[f] = fmaf(dd, dd, acc[f]);
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1)
#pragma unroll
    for (int f = 0; f < DP; ++f) acc[f] += __shfl_xor_sync(0xffffffffu, acc[f], o);
  dist[0] = dist[1] = 0.f;
#pragma unroll
  for (int f = 0; f < DP; ++f)
    if (f < ix.D && lane == f) dist[0] = sqrtf(acc[f]);
}

// Lower bound of dist_d from segment means (piecewise aggregate
// approximation): for 16-point segments of both windows,
//   sum_t (z_a - z_b)^2 >= sum_k 16 (mean_k z_a - mean_k z_b)^2
// (Cauchy-Schwarz on every segment; the points after the last full
// segment are left out, which only lowers the bound), and the sum of the d
// smallest per-dim bounds is below dist_d.  Reads w/16 rows per window.
template <int DP>
__device__ __forceinline__ float dist_d_lower_bound(const Index& ix, uint32_t a, uint32_t b, int d) {
  const int lane = threadIdx.x & 31;
  float m0a[DP], m1a[DP], isa[DP], m0b[DP], m1b[DP], isb[DP], acc[DP];
  load_stats<DP>(ix, a, m0a, m1a, isa);
  load_stats<DP>(ix, b, m0b, m1b, isb);
#pragma unroll
  for (int f = 0; f < DP; ++f) acc[f] = 0.f;
  const int segs = ix.w / 16;
  for (int k = lane; k < segs; k += 32) {
    float ua[DP], ub[DP];
    load_row<DP>(ix.smT, int64_t(a) + 16 * k, ua);
    load_row<DP>(ix.smT, int64_t(b) + 16 * k, ub);
#pragma unroll
    for (int f = 0; f < DP; ++f) {
      const float za = ((ua[f] - m0a[f]) - m1a[f]) * isa[f];
      const float zb = ((ub[f] - m0b[f]) - m1b[f]) * isb[f];
      const float dd = za - zb;
      acc[f] = fmaf(dd, dd, acc[f]);
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1)
#pragma unroll
    for (int f = 0; f < DP; ++f) acc[f] += __shfl_xor_sync(0xffffffffu, acc[f], o);
  float lb[DP];
#pragma unroll
  for (int f = 0; f < DP; ++f) lb[f] = f < ix.D ? sqrtf(16.f * acc[f]) : INFINITY;
  return sum_d_smallest<DP>(lb, ix.D, d);
}

// One warp per candidate event (each warp a contiguous range of events):
// distances; a pair with dist_d < tau is recorded (with its repetition) and
// offered to the set of close pairs.
// DM: dims held per lane (0 = any D); PM: the point-major copies (DP = DM)
template <int DM, bool PM, bool LO>
__global__ void __launch_bounds__(256)
k_verify_events(Index ix, int d, HashSet hs, const Event* __restrict__ ev,
                unsigned long long* __restrict__ counters, uint64_t ev_cap, float tau,
                PairRec* __restrict__ rec, uint64_t rec_cap) {
  const int lane = threadIdx.x & 31;
  uint64_t cnt = counters[0];
  if (cnt > ev_cap) cnt = ev_cap;
  const uint64_t nw = uint64_t(gridDim.x) * (blockDim.x >> 5);
  const uint64_t w = (blockIdx.x * uint64_t(blockDim.x) + threadIdx.x) >> 5;
  const uint64_t q0 = cnt * w / nw, q1 = cnt * (w + 1) / nw;
  for (uint64_t q = q0; q < q1; ++q) {
    const Event e = ev[q];
    if (PM && ix.smT) {
      const float lb = dist_d_lower_bound<(PM ? DM : 4)>(ix, e.a, e.b, d);
      if (lb > tau * (1.f + 1e-3f) + 1e-3f) {          // provably not below tau
        if (lane == 0) atomicAdd(&counters[3], 1ull);
        continue;
      }
    }
    float dist[2];
    if (PM) pair_distances_pm<(PM ? DM : 4), LO>(ix, e.a, e.b, dist);
    else if (DM > 0) pair_distances_fast<(DM > 0 ? DM : 1)>(ix, e.a, e.b, dist);
    else pair_distances<float>(ix, e.a, e.b, dist);
    VerifyOut v = select_d<float>(dist, ix.D, d);
    if (lane != 0) continue;
    if (!(float(v.dist_d) < tau)) {
      atomicAdd(&counters[4], 1ull);
      continue;
    }
    const unsigned long long pos = atomicAdd(&counters[1], 1ull);
    if (pos < rec_cap) {
      PairRec r;
      r.a = e.a;
      r.b = e.b;
      r.j = e.j;
      r.dist_d = float(v.dist_d);
      r.dist_max = float(v.dist_max);
      r.pad = 0;
      r.dims = v.mask;
      rec[pos] = r;
    }
    const uint64_t key = (uint64_t(e.a) << 32) | e.b;
    uint64_t h = set_hash(key) & (hs.cap - 1);
    for (int probe = 0; probe < kSetMaxProbe; ++probe) {
      uint64_t cur = hs.keys[h];
      if (cur == key) break;
      if (cur == kSetEmpty) {
        cur = atomicCAS(reinterpret_cast<unsigned long long*>(&hs.keys[h]), kSetEmpty, key);
        if (cur == kSetEmpty) {
          atomicAdd(&counters[2], 1ull);
          break;
        }
        if (cur == key) break;
      }
      h = (h + 1) & (hs.cap - 1);
    }
  }
}

__global__ void __launch_bounds__(256)
k_verify_pairs(Index ix, int d, const uint64_t* __restrict__ pairs, int64_t m, int fp64,
               double* __restrict__ per_dim, double* __restrict__ dist_d,
               uint64_t* __restrict__ dims) {
  const int lane = threadIdx.x & 31;
  const int64_t nw = int64_t(gridDim.x) * (blockDim.x >> 5);
  for (int64_t q = (blockIdx.x * int64_t(blockDim.x) + threadIdx.x) >> 5; q < m; q += nw) {
    const uint32_t a = uint32_t(pairs[q] >> 32), b = uint32_t(pairs[q]);
    VerifyOut v;
    double dd[2];
    if (fp64) {
      double dist[2];
      pair_distances<double>(ix, a, b, dist);
      v = select_d<double>(dist, ix.D, d);
      dd[0] = dist[0];
      dd[1] = dist[1];
    } else {
      float dist[2];
      pair_distances<float>(ix, a, b, dist);
      v = select_d<float>(dist, ix.D, d);
      dd[0] = dist[0];
      dd[1] = dist[1];
    }
    if (per_dim) {
      if (lane < ix.D) per_dim[q * ix.D + lane] = dd[0];
      if (lane + 32 < ix.D) per_dim[q * ix.D + lane + 32] = dd[1];
    }
    if (lane == 0) {
      if (dist_d) dist_d[q] = v.dist_d;
      if (dims) dims[q] = v.mask;
    }
  }
}

// ---- all pairs ------------------------------------------------------------

// A pair whose approximate dist_d lies in (rc.lo, thr]: appended (with its
// approximate distance) while there is room, and counted in the histogram
// of (rc.lo, thr] either way.
__device__ __forceinline__ void record_pair(const ApRec& rc, int64_t a, int64_t b, float dd) {
  // one counter atomic per group of converged lanes
  const unsigned act = __activemask();
  const int lane = threadIdx.x & 31, leader = __ffs(act) - 1;
  unsigned long long base = 0;
  if (lane == leader) base = atomicAdd(rc.count, (unsigned long long)__popc(act));
  base = __shfl_sync(act, base, leader);
  const unsigned long long pos = base + __popc(act & ((1u << lane) - 1u));
  if (pos < rc.cap) {
    rc.out[pos] = (uint64_t(a) << 32) | uint64_t(b);
    rc.out_d[pos] = dd;
  }
  if (rc.hist) {
    const float x = (dd - rc.lo) * rc.hscale;
    const int bin = x < float(kApBins - 1) ? int(fmaxf(x, 0.f)) : kApBins - 1;
    atomicAdd(&rc.hist[bin], 1u);
  }
}

// Diagonal steps between direct restarts: a restart costs w steps of a
// direct dot product, so it is amortised over many sliding steps (the
// float32 sliding sums drift by about sqrt(kSeg) roundings between
// restarts, far inside the 1% + 0.01 filter margin).
constexpr int kSeg = 2048;
constexpr int kRowSub = 256;     // row windows staged in shared memory at a time
constexpr int kDiagBlock = 256; // diagonals per CTA

__device__ __forceinline__ float xv(const float* xh, const float* xl, int64_t t) {
  return xl ? xh[t] + xl[t] : xh[t];
}

template <int DM, bool ROWMIN>
__global__ void __launch_bounds__(kDiagBlock)
k_allpairs(Index ix, int d, float thr, ApRec rc, float* __restrict__ rowmin, int64_t ybase) {
  const int64_t delta = int64_t(ix.excl) + 1 + (ybase + int64_t(blockIdx.y)) * kDiagBlock + threadIdx.x;
  const int64_t a0 = int64_t(blockIdx.x) * kSeg;
  if (delta >= ix.M || a0 >= ix.M - delta) return;
  const int64_t a1 = min(a0 + kSeg, ix.M - delta);
  const int D = ix.D, w = ix.w;
  const float wf = float(w), inv_w = 1.f / float(w);
  // per dim: sums of the two windows centred by ca / cb (sliding), and of
  // their products
  float qt[DM], s1a[DM], s2a[DM], s1b[DM], s2b[DM], ca[DM], cb[DM];
#pragma unroll
  for (int f = 0; f < DM; ++f) {
    qt[f] = s1a[f] = s2a[f] = s1b[f] = s2b[f] = ca[f] = cb[f] = 0.f;
    if (f < D) {
      const float* xh = ix.xs_hi + int64_t(f) * ix.n;
      const float* xl = ix.has_lo ? ix.xs_lo + int64_t(f) * ix.n : nullptr;
      ca[f] = ix.mu_hi[int64_t(f) * ix.M + a0];
      cb[f] = ix.mu_hi[int64_t(f) * ix.M + a0 + delta];
      float q = 0.f, u1 = 0.f, u2 = 0.f, v1 = 0.f, v2 = 0.f;
      for (int t = 0; t < w; ++t) {
        const float xa = xv(xh, xl, a0 + t) - ca[f], xb = xv(xh, xl, a0 + delta + t) - cb[f];
        q = fmaf(xa, xb, q);
        u1 += xa;
        u2 = fmaf(xa, xa, u2);
        v1 += xb;
        v2 = fmaf(xb, xb, v2);
      }
      qt[f] = q; s1a[f] = u1; s2a[f] = u2; s1b[f] = v1; s2b[f] = v2;
    }
  }
  for (int64_t a = a0; a < a1; ++a) {
    const int64_t b = a + delta;
    float dist[DM];
    int near = 0;
    bool unsure = false;
#pragma unroll
    for (int f = 0; f < DM; ++f) {
      dist[f] = INFINITY;
      if (f < D) {
        if (a > a0) {
          const float* xh = ix.xs_hi + int64_t(f) * ix.n;
          const float* xl = ix.has_lo ? ix.xs_lo + int64_t(f) * ix.n : nullptr;
          const float oa = xv(xh, xl, a - 1) - ca[f], ob = xv(xh, xl, b - 1) - cb[f];
          const float ia = xv(xh, xl, a + w - 1) - ca[f], ib = xv(xh, xl, b + w - 1) - cb[f];
          qt[f] = fmaf(ia, ib, fmaf(-oa, ob, qt[f]));
          s1a[f] += ia - oa;
          s2a[f] = fmaf(ia, ia, fmaf(-oa, oa, s2a[f]));
          s1b[f] += ib - ob;
          s2b[f] = fmaf(ib, ib, fmaf(-ob, ob, s2b[f]));
        }
        const float ma = s1a[f] * inv_w, mb = s1b[f] * inv_w;
        const float qa = s2a[f] * inv_w, qb = s2b[f] * inv_w;
        const float va = qa - ma * ma, vb = qb - mb * mb;
        const float cov = qt[f] * inv_w - ma * mb;
        // a variance lost to cancellation (a near-flat window): keep the pair
        // for the exact check
        const bool fa = !(va > 1e-4f * qa), fb = !(vb > 1e-4f * qb);
        float sq;
        if (fa || fb) {
          unsure = true;
          sq = 0.f;
        } else {
          sq = 2.f * wf * (1.f - cov * rsqrtf(va * vb));
        }
        dist[f] = sqrtf(fmaxf(sq, 0.f));
        near += dist[f] <= thr;
      }
    }
    if (ROWMIN) {
      float s = sum_d_smallest<DM>(dist, D, d);
      atomicMin(reinterpret_cast<int*>(rowmin + a), __float_as_int(s));
      atomicMin(reinterpret_cast<int*>(rowmin + b), __float_as_int(s));
    } else if (near >= d || unsure) {
      float s = unsure ? 0.f : sum_d_smallest<DM>(dist, D, d);
      if (s <= thr && s > rc.lo) record_pair(rc, a, b, s);
    }
  }
}

// Point-major series (D <= 8): the four time points a step touches are
// read as whole rows of DP dims (float4 loads); the window sums of both
// windows slide with the product sum, so no per-window statistic is read
// per step.
template <int DP, bool LO, bool ROWMIN>
__global__ void __launch_bounds__(kDiagBlock, 2)
k_allpairs_pm(Index ix, int d, float thr, ApRec rc, float* __restrict__ rowmin, int64_t ybase) {
  const int64_t delta = int64_t(ix.excl) + 1 + (ybase + int64_t(blockIdx.y)) * kDiagBlock + threadIdx.x;
  const int64_t a0 = int64_t(blockIdx.x) * kSeg;
  if (delta >= ix.M || a0 >= ix.M - delta) return;
  const int64_t a1 = min(a0 + kSeg, ix.M - delta);
  const int D = ix.D, w = ix.w;
  const float wf = float(w), inv_w = 1.f / float(w);
  const float* X = ix.xT;
  const float* XL = ix.xlT;
  float qt[DP], s1a[DP], s2a[DP], s1b[DP], s2b[DP], ca[DP], cb[DP];
#pragma unroll
  for (int f = 0; f < DP; ++f) {
    qt[f] = s1a[f] = s2a[f] = s1b[f] = s2b[f] = 0.f;
    ca[f] = f < D ? ix.mu_hi[int64_t(f) * ix.M + a0] : 0.f;
    cb[f] = f < D ? ix.mu_hi[int64_t(f) * ix.M + a0 + delta] : 0.f;
  }
  for (int t = 0; t < w; ++t) {
    float xa[DP], xb[DP];
    load_row<DP>(X, a0 + t, xa);
    load_row<DP>(X, a0 + delta + t, xb);
    if (LO) {
      float ya[DP], yb[DP];
      load_row<DP>(XL, a0 + t, ya);
      load_row<DP>(XL, a0 + delta + t, yb);
#pragma unroll
      for (int f = 0; f < DP; ++f) { xa[f] += ya[f]; xb[f] += yb[f]; }
    }
#pragma unroll
    for (int f = 0; f < DP; ++f) {
      const float u = xa[f] - ca[f], v = xb[f] - cb[f];
      qt[f] = fmaf(u, v, qt[f]);
      s1a[f] += u;
      s2a[f] = fmaf(u, u, s2a[f]);
      s1b[f] += v;
      s2b[f] = fmaf(v, v, s2b[f]);
    }
  }
  const float c0 = 1.f - thr * thr / (2.f * wf);
  const float c0sq = c0 * c0;
  for (int64_t a = a0; a < a1; ++a) {
    const int64_t b = a + delta;
    if (a > a0) {
      float oa[DP], ob[DP], ia[DP], ib[DP];
      load_row<DP>(X, a - 1, oa);
      load_row<DP>(X, b - 1, ob);
      load_row<DP>(X, a + w - 1, ia);
      load_row<DP>(X, b + w - 1, ib);
      if (LO) {
        float y[DP];
        load_row<DP>(XL, a - 1, y);
#pragma unroll
        for (int f = 0; f < DP; ++f) oa[f] += y[f];
        load_row<DP>(XL, b - 1, y);
#pragma unroll
        for (int f = 0; f < DP; ++f) ob[f] += y[f];
        load_row<DP>(XL, a + w - 1, y);
#pragma unroll
        for (int f = 0; f < DP; ++f) ia[f] += y[f];
        load_row<DP>(XL, b + w - 1, y);
#pragma unroll
        for (int f = 0; f < DP; ++f) ib[f] += y[f];
      }
#pragma unroll
      for (int f = 0; f < DP; ++f) {
        const float uo = oa[f] - ca[f], vo = ob[f] - cb[f];
        const float ui = ia[f] - ca[f], vi = ib[f] - cb[f];
        qt[f] = fmaf(ui, vi, fmaf(-uo, vo, qt[f]));
        s1a[f] += ui - uo;
        s2a[f] = fmaf(ui, ui, fmaf(-uo, uo, s2a[f]));
        s1b[f] += vi - vo;
        s2b[f] = fmaf(vi, vi, fmaf(-vo, vo, s2b[f]));
      }
    }
    // dist_f <= thr  <=>  corr >= c0 = 1 - thr^2 / 2w  <=>  C >= c0 sqrt(VA VB)
    // with C = w QT - S1a S1b, VA = w S2a - S1a^2 (sums of the centred windows)
    int near = 0;
    bool unsure = false;
    unsigned nmask = 0;
#pragma unroll
    for (int f = 0; f < DP; ++f) {
      if (f < D) {
        const float VA = fmaf(wf, s2a[f], -s1a[f] * s1a[f]);
        const float VB = fmaf(wf, s2b[f], -s1b[f] * s1b[f]);
        const float Cv = fmaf(wf, qt[f], -s1a[f] * s1b[f]);
        const bool flat = !(VA > 1e-4f * wf * s2a[f]) || !(VB > 1e-4f * wf * s2b[f]);
        unsure |= flat;
        const bool ok = c0 <= 0.f || (Cv > 0.f && Cv * Cv >= c0sq * VA * VB);
        near += ok;
        nmask |= unsigned(ok) << f;
      }
    }
    float dist[DP];
    if (ROWMIN || near >= d) {
#pragma unroll
      for (int f = 0; f < DP; ++f) {
        dist[f] = INFINITY;
        if (f < D) {
          const float VA = fmaf(wf, s2a[f], -s1a[f] * s1a[f]);
          const float VB = fmaf(wf, s2b[f], -s1b[f] * s1b[f]);
          const float Cv = fmaf(wf, qt[f], -s1a[f] * s1b[f]);
          const float sq = (VA > 0.f && VB > 0.f) ? 2.f * wf * (1.f - Cv * rsqrtf(VA * VB)) : 0.f;
          dist[f] = sqrtf(fmaxf(sq, 0.f));
        }
      }
    }
    (void)nmask;
    if (ROWMIN) {
      float sm = sum_d_smallest<DP>(dist, D, d);
      atomicMin(reinterpret_cast<int*>(rowmin + a), __float_as_int(sm));
      atomicMin(reinterpret_cast<int*>(rowmin + b), __float_as_int(sm));
    } else if (near >= d || unsure) {
      const float sm = unsure ? 0.f : sum_d_smallest<DP>(dist, D, d);
      if (sm <= thr && sm > rc.lo) record_pair(rc, a, b, sm);
    }
  }
}

// Point-major, block-shared rows: all diagonals of a block share the row
// windows a in [a0, a0 + kSeg).  The rows are staged in shared memory
// kRowSub at a time (small stages leave room for three CTAs per SM;
// centred by the first row window's mean of the stage,
// with their sliding sums); each thread keeps the column sums and the
// cross product of its diagonal and carries them across stages, re-centred
// on the new row and column means, so a direct restart (w steps) is paid
// once per kSeg steps.
template <int DP, bool ROWMIN>
__global__ void __launch_bounds__(kDiagBlock, DP <= 8 ? 3 : 2)
k_allpairs_rows(Index ix, int d, float thr, ApRec rc, float* __restrict__ rowmin, int64_t ybase) {
  extern __shared__ float ap_smem[];
  const int w = ix.w, D = ix.D;
  const int64_t a0 = int64_t(blockIdx.x) * kSeg;
  const int64_t dlo = int64_t(ix.excl) + 1 + (ybase + int64_t(blockIdx.y)) * kDiagBlock;
  if (dlo >= ix.M || a0 >= ix.M - dlo) return;                  // block-uniform
  const int64_t delta = dlo + threadIdx.x;
  const bool live = delta < ix.M && a0 < ix.M - delta;
  const int64_t a1 = live ? min(a0 + kSeg, ix.M - delta) : a0;
  const int64_t nrow = min(int64_t(kSeg), ix.M - dlo - a0);     // row windows this block needs
  // rowx[t] = point aS - 1 + t of the stage starting at row aS, centred
  float* rowx = ap_smem;                                        // [kRowSub + w][DP]
  float* sa1 = rowx + (kRowSub + w) * DP;                       // [kRowSub][DP] row sums
  float* sa2 = sa1 + kRowSub * DP;                              // [kRowSub][DP] w^2 var (-1: unreliable)
  float* cav = sa2 + kRowSub * DP;                              // [2][DP] row centring, by stage parity
  float* sprev = cav + 2 * DP;                                  // [DP] sum of row window aS - 1
  // per-warp queue of candidate pairs: state (qt, s1b, s2b per dim),
  // row and unsure flag, column window
  constexpr int QS = 3 * DP + 2;
  float* qall = sprev + DP;                                     // [warps][32][QS]
  uint32_t* qmeta = reinterpret_cast<uint32_t*>(qall + (kDiagBlock / 32) * 32 * QS);
  uint32_t* qcol = qmeta + kDiagBlock;
  __shared__ int rflag[kRowSub];                                // row window unreliable in some dim
  const float* X = ix.xT;
  constexpr int DH = DP / 2;
  const float wf = float(w);
  const float2 wf2 = make_float2(wf, wf);
  const float2* row2 = reinterpret_cast<const float2*>(rowx);
  const float2* sa1_2 = reinterpret_cast<const float2*>(sa1);
  const float2* sa2_2 = reinterpret_cast<const float2*>(sa2);
  // the per-step arithmetic runs on pairs of dims with the packed
  // two-lane float32 instructions (same rounding as the scalar ones)
  float2 qt[DH], s1b[DH], s2b[DH], ncb[DH];
#pragma unroll
  for (int p = 0; p < DH; ++p) {
    qt[p] = s1b[p] = s2b[p] = make_float2(0.f, 0.f);
    const int f0 = 2 * p, f1 = 2 * p + 1;
    ncb[p] = make_float2(live && f0 < D ? -ix.mu_hi[int64_t(f0) * ix.M + a0 + delta] : 0.f,
                         live && f1 < D ? -ix.mu_hi[int64_t(f1) * ix.M + a0 + delta] : 0.f);
  }
  // Necessary conditions of dist_d <= thr on the sorted per-dim distances
  // x(1) <= x(2) <= ...: x(1) <= thr / d and x(d) <= thr; with more than 8
  // dims (where d reaches 3..6) also x(2) <= thr / (d - 1).  The other
  // middle ones, x(i) <= thr / (d - i + 1), reject few more pairs than they
  // cost.  dist_f <= t  <=>  corr >= c = 1 - t^2 / 2w  <=>  C >= c sqrt(VA VB)
  // <=>  C |C| >= c |c| VA VB (x -> x |x| is monotone).
  constexpr bool kMid = DP >= 16;
  const float t1 = thr / float(d), t2 = d >= 2 ? thr / float(d - 1) : thr;
  const float c1 = 1.f - t1 * t1 / (2.f * wf), c2 = 1.f - t2 * t2 / (2.f * wf);
  const float cd = 1.f - thr * thr / (2.f * wf);
  const float2 k1 = make_float2(c1 * fabsf(c1), c1 * fabsf(c1));
  const float2 k2 = make_float2(c2 * fabsf(c2), c2 * fabsf(c2));
  const float2 kd = make_float2(cd * fabsf(cd), cd * fabsf(cd));
  const uint32_t need2 = d >= 2 ? 2u : 1u;
  const float2 flat = make_float2(1e-4f * wf, 1e-4f * wf);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  float* qst = qall + warp * 32 * QS;
  uint32_t* qm = qmeta + warp * 32;
  uint32_t* qc = qcol + warp * 32;
  int64_t aS = a0;                  // first row of the current stage
  // distances of queued pairs, one per lane (lanes below count)
  auto drain = [&](int count) {
    __syncwarp();
    if (lane < count) {
      const float* st = qst + lane * QS;
      const int r = int(qm[lane] >> 1);
      const bool uns = (qm[lane] & 1u) != 0;
      float dist[DP];
#pragma unroll
      for (int f = 0; f < DP; ++f) {
        dist[f] = INFINITY;
        if (f < D) {
          const float qf = st[f], s1 = st[DP + f], s2 = st[2 * DP + f];
          const float s1a = sa1[r * DP + f], VA = sa2[r * DP + f];
          const float VB = fmaf(wf, s2, -s1 * s1);
          const float Cv = fmaf(wf, qf, -s1a * s1);
          const float sq = (VA > 0.f && VB > 0.f) ? 2.f * wf * (1.f - Cv * rsqrtf(VA * VB)) : 0.f;
          dist[f] = sqrtf(fmaxf(sq, 0.f));
        }
      }
      const float sm = uns ? 0.f : sum_d_smallest<DP>(dist, D, d);
      if (sm <= thr && sm > rc.lo) record_pair(rc, aS + r, int64_t(qc[lane]), sm);
    }
    __syncwarp();
  };
  int qn = 0;                       // queued pairs of this warp (warp-uniform)
  for (int stage = 0; aS < a0 + nrow; ++stage, aS += kRowSub) {
    const int nsub = int(min(int64_t(kRowSub), a0 + nrow - aS));
    float* cnew = cav + (stage & 1) * DP;
    const float* cold = cav + ((stage & 1) ^ 1) * DP;
    __syncthreads();                // the previous stage is fully consumed
    if (threadIdx.x < DP) cnew[threadIdx.x] = threadIdx.x < D ? ix.mu_hi[int64_t(threadIdx.x) * ix.M + aS] : 0.f;
    __syncthreads();
    for (int q = threadIdx.x; q < (nsub + w) * DP; q += blockDim.x) {
      const int t = q / DP, f = q - t * DP;
      const int64_t pt = aS - 1 + t;
      rowx[q] = (f < D && pt >= 0) ? X[pt * DP + f] - cnew[f] : 0.f;
    }
    __syncthreads();
    if (threadIdx.x < DP) {                                     // one thread per dim slides the row sums
      const int f = threadIdx.x;
      float u1 = 0.f, u2 = 0.f;
      for (int t = 1; t <= w; ++t) {
        const float v = rowx[t * DP + f];
        u1 += v;
        u2 = fmaf(v, v, u2);
      }
      sprev[f] = u1 - rowx[w * DP + f] + rowx[f];               // window of row aS - 1
      // per row window: the sum and w^2 var (-1 when cancellation leaves it
      // unreliable: a near-flat window, always checked exactly)
      for (int r = 0; r < nsub; ++r) {
        if (r > 0) {
          const float o = rowx[r * DP + f], in = rowx[(r + w) * DP + f];
          u1 += in - o;
          u2 = fmaf(in, in, fmaf(-o, o, u2));
        }
        const float va = fmaf(wf, u2, -u1 * u1);
        sa1[r * DP + f] = u1;
        // padding dims: NaN, so that no test on them passes
        sa2[r * DP + f] = f >= D ? __int_as_float(0x7fc00000) : (va > 1e-4f * wf * u2 ? va : -1.f);
      }
    }
    __syncthreads();
    for (int r = threadIdx.x; r < nsub; r += blockDim.x) {
      int u = 0;
      for (int f = 0; f < D; ++f) u |= sa2[r * DP + f] < 0.f;
      rflag[r] = u;
    }
    __syncthreads();
    if (stage == 0) {
      // direct start: rows window a0 against column window a0 + delta
      for (int t = 0; t < (live ? w : 0); ++t) {
        float xb[DP];
        load_row<DP>(X, a0 + delta + t, xb);
#pragma unroll
        for (int p = 0; p < DH; ++p) {
          const float2 u = row2[(t + 1) * DH + p];
          const float2 v = __fadd2_rn(make_float2(xb[2 * p], xb[2 * p + 1]), ncb[p]);
          qt[p] = __ffma2_rn(u, v, qt[p]);
          s1b[p] = __fadd2_rn(s1b[p], v);
          s2b[p] = __ffma2_rn(v, v, s2b[p]);
        }
      }
    } else if (aS - 1 < a1) {
      // the state holds row window aS - 1 and column window aS - 1 + delta:
      // re-centre the rows on this stage's mean (qt += (c_old - c_new) s1b),
      // then the columns on that column window's mean (v' = v - dc)
#pragma unroll
      for (int p = 0; p < DH; ++p) {
        const int f0 = 2 * p, f1 = 2 * p + 1;
        const float2 dr = make_float2(cold[f0] - cnew[f0], cold[f1] - cnew[f1]);
        qt[p] = __ffma2_rn(dr, s1b[p], qt[p]);
        const float2 cbn = make_float2(f0 < D ? ix.mu_hi[int64_t(f0) * ix.M + aS - 1 + delta] : 0.f,
                                       f1 < D ? ix.mu_hi[int64_t(f1) * ix.M + aS - 1 + delta] : 0.f);
        const float2 dc = make_float2(cbn.x + ncb[p].x, cbn.y + ncb[p].y);
        const float2 sp = make_float2(sprev[f0], sprev[f1]);
        qt[p] = __ffma2_rn(make_float2(-dc.x, -dc.y), sp, qt[p]);
        s2b[p] = __ffma2_rn(make_float2(wf * dc.x, wf * dc.y), dc,
                            __ffma2_rn(make_float2(-2.f * dc.x, -2.f * dc.y), s1b[p], s2b[p]));
        s1b[p] = __ffma2_rn(make_float2(-wf, -wf), dc, s1b[p]);
        ncb[p] = make_float2(-cbn.x, -cbn.y);
      }
    }
    // every lane runs the stage's row count, so that the warp stays converged
    for (int r = 0; r < nsub; ++r) {
      const int64_t a = aS + r;
      const int64_t b = a + delta;
      const bool act = a < a1;
      if (act && (r > 0 || stage > 0)) {
        float ob[DP], ib[DP];
        load_row<DP>(X, b - 1, ob);
        load_row<DP>(X, b + w - 1, ib);
#pragma unroll
        for (int p = 0; p < DH; ++p) {
          const float2 uo = row2[r * DH + p], ui = row2[(r + w) * DH + p];
          const float2 vo = __fadd2_rn(make_float2(ob[2 * p], ob[2 * p + 1]), ncb[p]);
          const float2 vi = __fadd2_rn(make_float2(ib[2 * p], ib[2 * p + 1]), ncb[p]);
          qt[p] = __ffma2_rn(ui, vi, __ffma2_rn(make_float2(-uo.x, -uo.y), vo, qt[p]));
          s1b[p] = __fadd2_rn(s1b[p], __fadd2_rn(vi, make_float2(-vo.x, -vo.y)));
          s2b[p] = __ffma2_rn(vi, vi, __ffma2_rn(make_float2(-vo.x, -vo.y), vo, s2b[p]));
        }
      }
      uint32_t cnt = 0;            // tests passed: byte 0 x(1), byte 1 x(2), high half x(d)
      bool unsure = rflag[r] != 0;
#pragma unroll
      for (int p = 0; p < DH; ++p) {
        const float2 s1a = sa1_2[r * DH + p], VA = sa2_2[r * DH + p];
        const float2 VB = __ffma2_rn(wf2, s2b[p], __fmul2_rn(make_float2(-s1b[p].x, -s1b[p].y), s1b[p]));
        const float2 Cv = __ffma2_rn(wf2, qt[p], __fmul2_rn(make_float2(-s1a.x, -s1a.y), s1b[p]));
        const float2 P = __fmul2_rn(VA, VB);
        const float2 S = __fmul2_rn(Cv, make_float2(fabsf(Cv.x), fabsf(Cv.y)));
        const float2 T1 = __fmul2_rn(k1, P), Td = __fmul2_rn(kd, P);
        const float2 FB = __fmul2_rn(flat, s2b[p]);
        unsure |= (VB.x < FB.x) | (VB.y < FB.y);
        cnt += (S.x >= T1.x) + (S.y >= T1.y) + ((S.x >= Td.x) + (S.y >= Td.y)) * 65536u;
        if constexpr (kMid) {
          const float2 T2 = __fmul2_rn(k2, P);
          cnt += ((S.x >= T2.x) + (S.y >= T2.y)) * 256u;
        }
      }
      if (!ROWMIN) {
        const bool cand = act && (unsure || ((cnt & 255u) >= 1u && (!kMid || ((cnt >> 8) & 255u) >= need2) &&
                                             (cnt >> 16) >= uint32_t(d)));
        const unsigned m = __ballot_sync(0xffffffffu, cand);
        if (!m) continue;
        const int n = __popc(m);
        if (qn + n > 32) {
          drain(qn);
          qn = 0;
        }
        if (cand) {
          const int pos = qn + __popc(m & ((1u << lane) - 1u));
          float2* st = reinterpret_cast<float2*>(qst + pos * QS);
#pragma unroll
          for (int p = 0; p < DH; ++p) {
            st[p] = qt[p];
            st[DH + p] = s1b[p];
            st[2 * DH + p] = s2b[p];
          }
          qm[pos] = (uint32_t(r) << 1) | (unsure ? 1u : 0u);
          qc[pos] = uint32_t(b);
        }
        qn += n;
        if (qn == 32) {
          drain(32);
          qn = 0;
        }
        continue;
      }
      if (!act) continue;
      float dist[DP];
#pragma unroll
      for (int f = 0; f < DP; ++f) {
        dist[f] = INFINITY;
        if (f < D) {
          const float qf = (f & 1) ? qt[f >> 1].y : qt[f >> 1].x;
          const float s1 = (f & 1) ? s1b[f >> 1].y : s1b[f >> 1].x;
          const float s2 = (f & 1) ? s2b[f >> 1].y : s2b[f >> 1].x;
          const float s1a = sa1[r * DP + f], VA = sa2[r * DP + f];
          const float VB = fmaf(wf, s2, -s1 * s1);
          const float Cv = fmaf(wf, qf, -s1a * s1);
          const float sq = (VA > 0.f && VB > 0.f) ? 2.f * wf * (1.f - Cv * rsqrtf(VA * VB)) : 0.f;
          dist[f] = sqrtf(fmaxf(sq, 0.f));
        }
      }
      const float sm = sum_d_smallest<DP>(dist, D, d);
      atomicMin(reinterpret_cast<int*>(rowmin + a), __float_as_int(sm));
      atomicMin(reinterpret_cast<int*>(rowmin + b), __float_as_int(sm));
    }
    if (!ROWMIN) {                  // queued pairs refer to this stage's rows
      drain(qn);
      qn = 0;
    }
  }
}

// Row-staged sweep with the threshold test on window statistics (float32
// input, D <= 16, not the row minima).  The state of a diagonal is what the
// rows kernel above slides, less the column sums of squares: the cross
// product qt = sum (x_a - c_a)(x_b - c_b) of the row window a and the
// column window b = a + delta, each centred on a constant (c_a per stage,
// c_b per diagonal and stage), and the column sum s1b = sum (x_b - c_b).
// The identity
//   sum (x_a - mu_a)(x_b - mu_b) = qt - (mu_a - c_a) s1b  =: u
// gives corr = u / (w sigma_a sigma_b), so for sigma > 0
//   dist_f <= t  <=>  corr >= c(t) = 1 - t^2 / 2w  <=>  u / sigma_b >= c(t) w sigma_a.
// mu_a - c_a and w sigma_a come per staged row from the float64 window
// statistics, 1/sigma_b per column from the point-major table isT, so a
// pair and dim costs one FMA (u), one more (v = u / sigma_b) and one FMA
// per threshold whose sign bit is counted: the necessary conditions of the
// rows kernel (x(1) <= thr/d, x(d) <= thr, with more than 8 dims also
// x(2) <= thr/(d-1)).  Padding dims carry qt = -1 and 1/sigma = 1, so
// every test on them fails.  A pair whose row or column window cannot be
// tested reliably in float32 (flat, or its centring offset large against
// its sigma: rflag per stage, cflag per column) is always a candidate.
// Candidates go to a per-warp queue with their v per dim; their distances
// are computed 32 at a time.
constexpr int kRowSub3 = 256;

// One block of the sweep: row windows [bx kSeg, bx kSeg + kSeg), diagonals
// from eps + 1 + by kDiagBlock; RS rows staged at a time.
template <int DP, int RS>
__device__ __forceinline__ void rows3_body(const Index& ix, int d, float thr, const ApRec& rc,
                                           int64_t bx, int64_t by) {
  constexpr int DH = DP / 2;
  constexpr bool kMid = DP >= 16;
  constexpr int QS = DP + 2;                                    // queued: v per dim, row/unsure, column
  extern __shared__ float ap_smem[];
  const int w = ix.w, D = ix.D;
  const int64_t a0 = bx * kSeg;
  const int64_t dlo = int64_t(ix.excl) + 1 + by * kDiagBlock;
  if (dlo >= ix.M || a0 >= ix.M - dlo) return;                  // block-uniform
  const int64_t delta = dlo + threadIdx.x;
  const bool live = delta < ix.M && a0 < ix.M - delta;
  const int64_t a1 = live ? min(a0 + kSeg, ix.M - delta) : a0;
  const int64_t nrow = min(int64_t(kSeg), ix.M - dlo - a0);
  float* rowx = ap_smem;                                        // [RS][DH] {-(x_{a-1} - c_a) x2, x_{a+w-1} - c_a x2}
  float* rowc = rowx + RS * 2 * DP;                             // [RS][DH] {-(mu_a - c_a) x2, w sigma_a x2}
  float* cav = rowc + RS * 2 * DP;                              // [2][DP]
  float* sprev = cav + 2 * DP;                                  // [DP]
  float* qall = sprev + DP;                                     // [warps][32][QS]
  __shared__ int rflag[RS];
  const float* X = ix.xT;
  const float wf = float(w);
  const double wd = double(w);
  const float4* rowx4 = reinterpret_cast<const float4*>(rowx);
  const float4* rowc4 = reinterpret_cast<const float4*>(rowc);
  float2 qt[DH], s1b[DH], ncb[DH];
#pragma unroll
  for (int p = 0; p < DH; ++p) {
    const int f0 = 2 * p, f1 = 2 * p + 1;
    qt[p] = make_float2(f0 < D ? 0.f : -1.f, f1 < D ? 0.f : -1.f);
    s1b[p] = make_float2(0.f, 0.f);
    ncb[p] = make_float2(live && f0 < D ? -ix.mu_hi[int64_t(f0) * ix.M + a0 + delta] : 0.f,
                         live && f1 < D ? -ix.mu_hi[int64_t(f1) * ix.M + a0 + delta] : 0.f);
  }
  const float t1 = thr / float(d), t2 = d >= 2 ? thr / float(d - 1) : thr;
  const float c1 = 1.f - t1 * t1 / (2.f * wf), c2 = 1.f - t2 * t2 / (2.f * wf);
  const float cd = 1.f - thr * thr / (2.f * wf);
  const float2 nc1 = make_float2(-c1, -c1), nc2 = make_float2(-c2, -c2), ncd = make_float2(-cd, -cd);
  const int need2 = d >= 2 ? 2 : 1;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  float* qst = qall + warp * 32 * QS;
  int64_t aS = a0;
  auto drain = [&](int count) {
    __syncwarp();
    if (lane < count) {
      const float* st = qst + lane * QS;
      const uint32_t meta = __float_as_uint(st[DP]);
      const int r = int(meta >> 1);
      const bool uns = (meta & 1u) != 0;
      float dist[DP];
#pragma unroll
      for (int f = 0; f < DP; ++f) {
        dist[f] = INFINITY;
        if (f < D) {
          const float wsa = rowc[(r * DH + (f >> 1)) * 4 + 2 + (f & 1)];
          const float corr = st[f] / wsa;
          dist[f] = sqrtf(fmaxf(2.f * wf * (1.f - corr), 0.f));
        }
      }
      const float sm = uns ? 0.f : sum_d_smallest<DP>(dist, D, d);
      if (sm <= thr && sm > rc.lo) record_pair(rc, aS + r, int64_t(__float_as_uint(st[DP + 1])), sm);
    }
    __syncwarp();
  };
  int qn = 0;
  for (int stage = 0; aS < a0 + nrow; ++stage, aS += RS) {
    const int nsub = int(min(int64_t(RS), a0 + nrow - aS));
    float* cnew = cav + (stage & 1) * DP;
    const float* cold = cav + ((stage & 1) ^ 1) * DP;
    __syncthreads();                // the previous stage is fully consumed
    if (threadIdx.x < DP) {
      const int f = threadIdx.x;
      const float c = f < D ? ix.mu_hi[int64_t(f) * ix.M + aS] : 0.f;
      cnew[f] = c;
      sprev[f] = (f < D && aS >= 1) ? float(wd * (ix.mu[int64_t(f) * ix.M + aS - 1] - double(c))) : 0.f;
    }
    for (int r = threadIdx.x; r < RS; r += blockDim.x) rflag[r] = 0;
    __syncthreads();
    for (int q = threadIdx.x; q < nsub * DP; q += blockDim.x) {
      const int r = q / DP, f = q - r * DP;
      const int64_t a = aS + r;
      float* rcq = rowc + (r * DH + (f >> 1)) * 4 + (f & 1);
      float* rxq = rowx + (r * DH + (f >> 1)) * 4 + (f & 1);
      if (f < D) {
        const float c = cnew[f];
        rxq[0] = a >= 1 ? c - X[(a - 1) * DP + f] : 0.f;
        rxq[2] = X[(a + w - 1) * DP + f] - c;
        // unreliable (flat, or the centring offset large against sigma):
        // sigma^2 <= 1e-4 (sigma^2 + (mu - c)^2)
        const double m = ix.mu[int64_t(f) * ix.M + a], sg = ix.sig[int64_t(f) * ix.M + a];
        const double dm = m - double(c), v = sg * sg;
        const bool ok = v > 1e-4 * (v + dm * dm) && ix.inv_sig[int64_t(f) * ix.M + a] != 0.f;
        rcq[0] = ok ? float(-dm) : 0.f;
        rcq[2] = ok ? float(wd * sg) : 1.f;
        if (!ok) atomicOr(&rflag[r], 1);
      } else {
        rxq[0] = rxq[2] = 0.f;
        rcq[0] = 0.f;
        rcq[2] = 0.f;
      }
    }
    __syncthreads();
    if (stage == 0) {
      // direct start: row window a0 against column window a0 + delta
      for (int t = 0; t < (live ? w : 0); ++t) {
        float xa[DP], xb[DP];
        load_row<DP>(X, a0 + t, xa);                            // same address over the block
        load_row<DP>(X, a0 + delta + t, xb);
#pragma unroll
        for (int p = 0; p < DH; ++p) {
          const float2 u = make_float2(xa[2 * p] - cnew[2 * p], xa[2 * p + 1] - cnew[2 * p + 1]);
          const float2 v = __fadd2_rn(make_float2(xb[2 * p], xb[2 * p + 1]), ncb[p]);
          qt[p] = __ffma2_rn(u, v, qt[p]);
          s1b[p] = __fadd2_rn(s1b[p], v);
        }
      }
    } else if (aS - 1 < a1) {
      // the state holds row window aS - 1 and column window aS - 1 + delta:
      // re-centre the rows on this stage's constant, then the column on
      // that column window's mean
#pragma unroll
      for (int p = 0; p < DH; ++p) {
        const int f0 = 2 * p, f1 = 2 * p + 1;
        const float2 dr = make_float2(cold[f0] - cnew[f0], cold[f1] - cnew[f1]);
        qt[p] = __ffma2_rn(dr, s1b[p], qt[p]);
        const float2 cbn = make_float2(f0 < D ? ix.mu_hi[int64_t(f0) * ix.M + aS - 1 + delta] : 0.f,
                                       f1 < D ? ix.mu_hi[int64_t(f1) * ix.M + aS - 1 + delta] : 0.f);
        const float2 dc = make_float2(cbn.x + ncb[p].x, cbn.y + ncb[p].y);
        qt[p] = __ffma2_rn(make_float2(-dc.x, -dc.y), make_float2(sprev[f0], sprev[f1]), qt[p]);
        s1b[p] = __ffma2_rn(make_float2(-wf, -wf), dc, s1b[p]);
        ncb[p] = make_float2(-cbn.x, -cbn.y);
      }
    }
    for (int r = 0; r < nsub; ++r) {
      const int64_t a = aS + r;
      const int64_t b = a + delta;
      const bool act = a < a1;
      float isb[DP];
      int unsure = rflag[r];
      if (act) {
        if (r > 0 || stage > 0) {
          float ob[DP], ib[DP];
          load_col<DP>(X, b - 1, ob);
          load_col<DP>(X, b + w - 1, ib);
#pragma unroll
          for (int p = 0; p < DH; ++p) {
            const float4 xq = rowx4[r * DH + p];
            const float2 o = make_float2(ob[2 * p], ob[2 * p + 1]);
            const float2 i = make_float2(ib[2 * p], ib[2 * p + 1]);
            const float2 vo = __fadd2_rn(o, ncb[p]), vi = __fadd2_rn(i, ncb[p]);
            qt[p] = __ffma2_rn(make_float2(xq.z, xq.w), vi, __ffma2_rn(make_float2(xq.x, xq.y), vo, qt[p]));
            s1b[p] = __ffma2_rn(make_float2(-1.f, -1.f), o, __fadd2_rn(s1b[p], i));
          }
        }
        load_col<DP>(ix.isT, b, isb);
        unsure |= ix.cflag[b];
      } else {
#pragma unroll
        for (int f = 0; f < DP; ++f) isb[f] = 0.f;
      }
      uint32_t all1 = 0xffffffffu;  // sign bits of x(1)'s test: all set = no dim passes
      int negd = 0, neg2 = 0;       // dims failing x(d)'s and x(2)'s tests
      float2 v[DH];
#pragma unroll
      for (int p = 0; p < DH; ++p) {
        const float4 rq = rowc4[r * DH + p];
        const float2 u = __ffma2_rn(make_float2(rq.x, rq.y), s1b[p], qt[p]);
        v[p] = __fmul2_rn(u, make_float2(isb[2 * p], isb[2 * p + 1]));
        const float2 wsa = make_float2(rq.z, rq.w);
        const float2 e1 = __ffma2_rn(nc1, wsa, v[p]);
        const float2 ed = __ffma2_rn(ncd, wsa, v[p]);
        all1 &= __float_as_uint(e1.x) & __float_as_uint(e1.y);
        negd += int(__float_as_uint(ed.x) >> 31) + int(__float_as_uint(ed.y) >> 31);
        if constexpr (kMid) {
          const float2 e2 = __ffma2_rn(nc2, wsa, v[p]);
          neg2 += int(__float_as_uint(e2.x) >> 31) + int(__float_as_uint(e2.y) >> 31);
        }
      }
      const bool cand = act && (unsure || ((all1 >> 31) == 0u && DP - negd >= d &&
                                           (!kMid || DP - neg2 >= need2)));
      const unsigned m = __ballot_sync(0xffffffffu, cand);
      if (!m) continue;
      const int n = __popc(m);
      if (qn + n > 32) {
        drain(qn);
        qn = 0;
      }
      if (cand) {
        const int pos = qn + __popc(m & ((1u << lane) - 1u));
        float* st = qst + pos * QS;
#pragma unroll
        for (int p = 0; p < DH; ++p) {
          st[2 * p] = v[p].x;
          st[2 * p + 1] = v[p].y;
        }
        st[DP] = __uint_as_float((uint32_t(r) << 1) | (unsure ? 1u : 0u));
        st[DP + 1] = __uint_as_float(uint32_t(b));
      }
      qn += n;
      if (qn == 32) {
        drain(32);
        qn = 0;
      }
    }
    drain(qn);                      // queued pairs refer to this stage's rows
    qn = 0;
  }
}

// Row-staged sweep for 16 < D <= DW (point-major copy X [n][DW], float32
// input): the rows kernel above with the dims of each diagonal split over
// G = DW / 16 adjacent lanes, 16 dims each, so that every lane keeps the
// state of the D <= 16 form (cross products, column sums, column centring
// of its 16 dims).  The lanes of a diagonal add their threshold-test
// counts with shuffles; a candidate's state goes to a per-warp queue
// (one entry per diagonal, each lane writing its dims) and its distances
// are computed by one lane over all dims.  A stage stages only what its
// rows consume: the outgoing point a - 1 and the incoming point a + w - 1
// of each row window (2 kRowSub2 points per dim, whatever w is), and
// takes the row windows' centred sums from the float64 window statistics
// (sum w (mu - c), w^2 var w^2 sigma^2); the first row window's points,
// needed once per block for the direct start, are read from global memory.
constexpr int kRowSub2 = 96;

template <int DW, bool ROWMIN>
__global__ void __launch_bounds__(kDiagBlock, DW <= 32 ? 2 : 1)
k_allpairs_rows2(Index ix, const float* __restrict__ X, int d, float thr, ApRec rc,
                 float* __restrict__ rowmin, int64_t ybase) {
  constexpr int G = DW / 16;                 // lanes per diagonal
  constexpr int NDG = kDiagBlock / G;        // diagonals per block
  constexpr int DH = 8;                      // float2 pairs of dims per lane
  constexpr int DW2 = DW / 2;
  constexpr int RS = kRowSub2;
  constexpr int QS = 3 * DW + 2;             // queued state: qt, s1b, s2b per dim
  constexpr int QN = 32 / G;                 // queue entries per warp
  extern __shared__ float ap_smem[];
  const int w = ix.w, D = ix.D;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int g = threadIdx.x % G;
  const int f0 = 16 * g;                     // this lane's first dim
  const int64_t a0 = int64_t(blockIdx.x) * kSeg;
  const int64_t dlo = int64_t(ix.excl) + 1 + (ybase + int64_t(blockIdx.y)) * NDG;
  if (dlo >= ix.M || a0 >= ix.M - dlo) return;                  // block-uniform
  const int64_t delta = dlo + threadIdx.x / G;
  const bool live = delta < ix.M && a0 < ix.M - delta;
  const int64_t a1 = live ? min(a0 + kSeg, ix.M - delta) : a0;
  const int64_t nrow = min(int64_t(kSeg), ix.M - dlo - a0);
  float* outx = ap_smem;                                        // [RS][DW] point a - 1, centred
  float* inx = outx + RS * DW;                                  // [RS][DW] point a + w - 1, centred
  float* sa1 = inx + RS * DW;                                   // [RS][DW] centred row sums
  float* sa2 = sa1 + RS * DW;                                   // [RS][DW] w^2 var (-1: unreliable)
  float* cav = sa2 + RS * DW;                                   // [2][DW]
  float* sprev = cav + 2 * DW;                                  // [DW]
  float* qall = sprev + DW;                                     // [warps][QN][QS]
  uint32_t* qmeta = reinterpret_cast<uint32_t*>(qall + (kDiagBlock / 32) * QN * QS);
  uint32_t* qcol = qmeta + (kDiagBlock / 32) * QN;
  __shared__ int rflag[RS];
  const float wf = float(w);
  const double wd = double(w);
  const float2 wf2 = make_float2(wf, wf);
  const float2* out2 = reinterpret_cast<const float2*>(outx);
  const float2* in2 = reinterpret_cast<const float2*>(inx);
  const float2* sa1_2 = reinterpret_cast<const float2*>(sa1);
  const float2* sa2_2 = reinterpret_cast<const float2*>(sa2);
  float2 qt[DH], s1b[DH], s2b[DH], ncb[DH];
#pragma unroll
  for (int p = 0; p < DH; ++p) {
    qt[p] = s1b[p] = s2b[p] = make_float2(0.f, 0.f);
    const int fa = f0 + 2 * p, fb = fa + 1;
    ncb[p] = make_float2(live && fa < D ? -ix.mu_hi[int64_t(fa) * ix.M + a0 + delta] : 0.f,
                         live && fb < D ? -ix.mu_hi[int64_t(fb) * ix.M + a0 + delta] : 0.f);
  }
  // the necessary conditions of the rows kernel (x(1) <= thr/d, x(2) <=
  // thr/(d-1), x(d) <= thr on the sorted per-dim distances)
  const float t1 = thr / float(d), t2 = d >= 2 ? thr / float(d - 1) : thr;
  const float c1 = 1.f - t1 * t1 / (2.f * wf), c2 = 1.f - t2 * t2 / (2.f * wf);
  const float cd = 1.f - thr * thr / (2.f * wf);
  const float2 k1 = make_float2(c1 * fabsf(c1), c1 * fabsf(c1));
  const float2 k2 = make_float2(c2 * fabsf(c2), c2 * fabsf(c2));
  const float2 kd = make_float2(cd * fabsf(cd), cd * fabsf(cd));
  const uint32_t need2 = d >= 2 ? 2u : 1u;
  const float2 flat = make_float2(1e-4f * wf, 1e-4f * wf);
  float* qst = qall + warp * QN * QS;
  uint32_t* qm = qmeta + warp * QN;
  uint32_t* qc = qcol + warp * QN;
  int64_t aS = a0;
  // distances of queued diagonals, one per lane (lanes below count)
  auto drain = [&](int count) {
    __syncwarp();
    if (lane < count) {
      const float* st = qst + lane * QS;
      const int r = int(qm[lane] >> 1);
      const bool uns = (qm[lane] & 1u) != 0;
      float dist[DW];
#pragma unroll
      for (int f = 0; f < DW; ++f) {
        dist[f] = INFINITY;
        if (f < D) {
          const float qf = st[f], s1 = st[DW + f], s2 = st[2 * DW + f];
          const float s1a = sa1[r * DW + f], VA = sa2[r * DW + f];
          const float VB = fmaf(wf, s2, -s1 * s1);
          const float Cv = fmaf(wf, qf, -s1a * s1);
          const float sq = (VA > 0.f && VB > 0.f) ? 2.f * wf * (1.f - Cv * rsqrtf(VA * VB)) : 0.f;
          dist[f] = sqrtf(fmaxf(sq, 0.f));
        }
      }
      const float sm = uns ? 0.f : sum_d_smallest<DW>(dist, D, d);
      if (sm <= thr && sm > rc.lo) record_pair(rc, aS + r, int64_t(qc[lane]), sm);
    }
    __syncwarp();
  };
  int qn = 0;                       // queued diagonals of this warp (warp-uniform)
  for (int stage = 0; aS < a0 + nrow; ++stage, aS += RS) {
    const int nsub = int(min(int64_t(RS), a0 + nrow - aS));
    float* cnew = cav + (stage & 1) * DW;
    const float* cold = cav + ((stage & 1) ^ 1) * DW;
    __syncthreads();                // the previous stage is fully consumed
    if (threadIdx.x < DW) {
      const int f = threadIdx.x;
      const float c = f < D ? ix.mu_hi[int64_t(f) * ix.M + aS] : 0.f;
      cnew[f] = c;
      // centred sum of row window aS - 1 (re-centring of the carried state)
      sprev[f] = (f < D && aS >= 1) ? float(wd * (ix.mu[int64_t(f) * ix.M + aS - 1] - double(c))) : 0.f;
    }
    __syncthreads();
    for (int q = threadIdx.x; q < nsub * DW; q += blockDim.x) {
      const int r = q / DW, f = q - r * DW;
      const int64_t a = aS + r;
      if (f < D) {
        const float c = cnew[f];
        outx[q] = a >= 1 ? X[(a - 1) * DW + f] - c : 0.f;
        inx[q] = X[(a + w - 1) * DW + f] - c;
        // row window a centred on c: sum w (mu - c), w^2 var = w^2 sigma^2;
        // unreliable (near-flat) when sigma^2 <= 1e-4 (sigma^2 + (mu - c)^2)
        const double m = ix.mu[int64_t(f) * ix.M + a], sg = ix.sig[int64_t(f) * ix.M + a];
        const double dm = m - double(c), v = sg * sg;
        sa1[q] = float(wd * dm);
        sa2[q] = v > 1e-4 * (v + dm * dm) ? float(wd * wd * v) : -1.f;
      } else {
        outx[q] = inx[q] = sa1[q] = 0.f;
        sa2[q] = __int_as_float(0x7fc00000);      // padding dims: no test passes
      }
    }
    __syncthreads();
    for (int r = threadIdx.x; r < nsub; r += blockDim.x) {
      int u = 0;
      for (int f = 0; f < D; ++f) u |= sa2[r * DW + f] < 0.f;
      rflag[r] = u;
    }
    __syncthreads();
    if (stage == 0) {
      // direct start: row window a0 against column window a0 + delta
      for (int t = 0; t < (live ? w : 0); ++t) {
        float xa[16], xb[16];
        load_row<16>(X + f0, (a0 + t) * G, xa);                 // same address over the block
        load_row<16>(X + f0, (a0 + delta + t) * G, xb);
#pragma unroll
        for (int p = 0; p < DH; ++p) {
          const float2 u = make_float2(xa[2 * p] - cnew[f0 + 2 * p], xa[2 * p + 1] - cnew[f0 + 2 * p + 1]);
          const float2 v = __fadd2_rn(make_float2(xb[2 * p], xb[2 * p + 1]), ncb[p]);
          qt[p] = __ffma2_rn(u, v, qt[p]);
          s1b[p] = __fadd2_rn(s1b[p], v);
          s2b[p] = __ffma2_rn(v, v, s2b[p]);
        }
      }
    } else if (aS - 1 < a1) {
#pragma unroll
      for (int p = 0; p < DH; ++p) {
        const int fa = f0 + 2 * p, fb = fa + 1;
        const float2 dr = make_float2(cold[fa] - cnew[fa], cold[fb] - cnew[fb]);
        qt[p] = __ffma2_rn(dr, s1b[p], qt[p]);
        const float2 cbn = make_float2(fa < D ? ix.mu_hi[int64_t(fa) * ix.M + aS - 1 + delta] : 0.f,
                                       fb < D ? ix.mu_hi[int64_t(fb) * ix.M + aS - 1 + delta] : 0.f);
        const float2 dc = make_float2(cbn.x + ncb[p].x, cbn.y + ncb[p].y);
        const float2 sp = make_float2(sprev[fa], sprev[fb]);
        qt[p] = __ffma2_rn(make_float2(-dc.x, -dc.y), sp, qt[p]);
        s2b[p] = __ffma2_rn(make_float2(wf * dc.x, wf * dc.y), dc,
                            __ffma2_rn(make_float2(-2.f * dc.x, -2.f * dc.y), s1b[p], s2b[p]));
        s1b[p] = __ffma2_rn(make_float2(-wf, -wf), dc, s1b[p]);
        ncb[p] = make_float2(-cbn.x, -cbn.y);
      }
    }
    for (int r = 0; r < nsub; ++r) {
      const int64_t a = aS + r;
      const int64_t b = a + delta;
      const bool act = a < a1;
      if (act && (r > 0 || stage > 0)) {
        float ob[16], ib[16];
        load_row<16>(X + f0, (b - 1) * G, ob);
        load_row<16>(X + f0, (b + w - 1) * G, ib);
#pragma unroll
        for (int p = 0; p < DH; ++p) {
          const float2 uo = out2[r * DW2 + f0 / 2 + p], ui = in2[r * DW2 + f0 / 2 + p];
          const float2 vo = __fadd2_rn(make_float2(ob[2 * p], ob[2 * p + 1]), ncb[p]);
          const float2 vi = __fadd2_rn(make_float2(ib[2 * p], ib[2 * p + 1]), ncb[p]);
          qt[p] = __ffma2_rn(ui, vi, __ffma2_rn(make_float2(-uo.x, -uo.y), vo, qt[p]));
          s1b[p] = __fadd2_rn(s1b[p], __fadd2_rn(vi, make_float2(-vo.x, -vo.y)));
          s2b[p] = __ffma2_rn(vi, vi, __ffma2_rn(make_float2(-vo.x, -vo.y), vo, s2b[p]));
        }
      }
      uint32_t cnt = 0;            // tests passed: byte 0 x(1), byte 1 x(2), high half x(d)
      int unsure = 0;
#pragma unroll
      for (int p = 0; p < DH; ++p) {
        const float2 s1a = sa1_2[r * DW2 + f0 / 2 + p], VA = sa2_2[r * DW2 + f0 / 2 + p];
        const float2 VB = __ffma2_rn(wf2, s2b[p], __fmul2_rn(make_float2(-s1b[p].x, -s1b[p].y), s1b[p]));
        const float2 Cv = __ffma2_rn(wf2, qt[p], __fmul2_rn(make_float2(-s1a.x, -s1a.y), s1b[p]));
        const float2 P = __fmul2_rn(VA, VB);
        const float2 S = __fmul2_rn(Cv, make_float2(fabsf(Cv.x), fabsf(Cv.y)));
        const float2 T1 = __fmul2_rn(k1, P), T2 = __fmul2_rn(k2, P), Td = __fmul2_rn(kd, P);
        const float2 FB = __fmul2_rn(flat, s2b[p]);
        const int fa = f0 + 2 * p;
        unsure |= (fa < D && VB.x < FB.x) | (fa + 1 < D && VB.y < FB.y);
        cnt += (S.x >= T1.x) + (S.y >= T1.y) + ((S.x >= T2.x) + (S.y >= T2.y)) * 256u +
               ((S.x >= Td.x) + (S.y >= Td.y)) * 65536u;
      }
      // the diagonal's totals over its G lanes
#pragma unroll
      for (int o = 1; o < G; o <<= 1) {
        cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
        unsure |= __shfl_xor_sync(0xffffffffu, unsure, o);
      }
      unsure |= rflag[r];
      if (!ROWMIN) {
        const bool cand = act && (unsure || ((cnt & 255u) >= 1u && ((cnt >> 8) & 255u) >= need2 &&
                                             (cnt >> 16) >= uint32_t(d)));
        const unsigned m = __ballot_sync(0xffffffffu, cand);
        if (!m) continue;
        const int n = __popc(m) / G;                  // candidate diagonals of this step
        if (qn + n > QN) {
          drain(qn);
          qn = 0;
        }
        if (cand) {
          const int base = lane - g;                  // the diagonal's first lane
          const int pos = qn + __popc(m & ((1u << base) - 1u)) / G;
          float* st = qst + pos * QS;
#pragma unroll
          for (int p = 0; p < DH; ++p) {
            st[f0 + 2 * p] = qt[p].x;           st[f0 + 2 * p + 1] = qt[p].y;
            st[DW + f0 + 2 * p] = s1b[p].x;     st[DW + f0 + 2 * p + 1] = s1b[p].y;
            st[2 * DW + f0 + 2 * p] = s2b[p].x; st[2 * DW + f0 + 2 * p + 1] = s2b[p].y;
          }
          if (g == 0) {
            qm[pos] = (uint32_t(r) << 1) | (unsure ? 1u : 0u);
            qc[pos] = uint32_t(b);
          }
        }
        qn += n;
        if (qn == QN) {
          drain(QN);
          qn = 0;
        }
        continue;
      }
      // row minima: every pair's dist_d from all its dims (gathered on lane g = 0)
      float mine[16];
#pragma unroll
      for (int p = 0; p < DH; ++p) {
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const int f = f0 + 2 * p + h;
          const float qf = h ? qt[p].y : qt[p].x, s1 = h ? s1b[p].y : s1b[p].x, s2 = h ? s2b[p].y : s2b[p].x;
          const float s1a = sa1[r * DW + f], VA = sa2[r * DW + f];
          const float VB = fmaf(wf, s2, -s1 * s1);
          const float Cv = fmaf(wf, qf, -s1a * s1);
          const float sq = (VA > 0.f && VB > 0.f) ? 2.f * wf * (1.f - Cv * rsqrtf(VA * VB)) : 0.f;
          mine[2 * p + h] = f < D ? sqrtf(fmaxf(sq, 0.f)) : INFINITY;
        }
      }
      float dist[DW];
#pragma unroll
      for (int gg = 0; gg < G; ++gg) {
#pragma unroll
        for (int q = 0; q < 16; ++q) dist[16 * gg + q] = __shfl_sync(0xffffffffu, mine[q], lane - g + gg);
      }
      if (!act || g != 0) continue;
      const float sm = sum_d_smallest<DW>(dist, D, d);
      atomicMin(reinterpret_cast<int*>(rowmin + a), __float_as_int(sm));
      atomicMin(reinterpret_cast<int*>(rowmin + b), __float_as_int(sm));
    }
    if (!ROWMIN) {                  // queued diagonals refer to this stage's rows
      drain(qn);
      qn = 0;
    }
  }
}

// The sweep as a grid of blocks (x: row blocks, y: diagonal blocks from ybase).
template <int DP, int RS, int MINB>
__global__ void __launch_bounds__(kDiagBlock, MINB)
k_allpairs_rows3(Index ix, int d, float thr, ApRec rc, int64_t ybase) {
  rows3_body<DP, RS>(ix, d, thr, rc, int64_t(blockIdx.x), ybase + int64_t(blockIdx.y));
}

// The sweeps of several series in one persistent launch: each CTA takes
// (series, row block, diagonal block) items from a device queue in order
// (largest series first) until the queue is empty; an item is one block of
// the sweep above on that series' index, threshold and record buffers.
template <int DP, int RS, int MINB>
__global__ void __launch_bounds__(kDiagBlock, MINB)
k_allpairs_rows3_batch(const SweepJob* __restrict__ jobs, const SweepItem* __restrict__ items,
                       int nitems, int* __restrict__ next) {
  __shared__ int cur;
  for (;;) {
    __syncthreads();                // every thread has read the previous item
    if (threadIdx.x == 0) cur = atomicAdd(next, 1);
    __syncthreads();
    const int it = cur;
    if (it >= nitems) return;       // block-uniform
    const SweepItem q = items[it];
    const SweepJob& j = jobs[q.job];
    rows3_body<DP, RS>(j.ix, j.d, j.thr, j.rc, int64_t(q.bx), int64_t(q.by));
  }
}

// The statistics form of the threshold test (the rows3 kernel above) for
// wide series, 16 < D <= DW (point-major copy X [n][DW], float32 input),
// with the dims of a diagonal split over G = DW / 16 adjacent lanes as in
// the rows2 kernel.  Each lane slides qt and s1b of its 16 dims and tests
// them against its row factors and the column table isW; the lanes of a
// diagonal combine their sign-bit counts with shuffles.  A candidate's v
// per dim goes to a per-warp queue (one entry per diagonal, each lane
// writing its dims) and its distances are computed by one lane.
template <int DW>
__global__ void __launch_bounds__(kDiagBlock, DW <= 32 ? 2 : 1)
k_allpairs_rows4(Index ix, const float* __restrict__ X, int d, float thr, ApRec rc, int64_t ybase) {
  constexpr int G = DW / 16;                 // lanes per diagonal
  constexpr int NDG = kDiagBlock / G;        // diagonals per block
  constexpr int DH = 8;                      // float2 pairs of dims per lane
  constexpr int DW2 = DW / 2;
  constexpr int RS = kRowSub2;
  constexpr int QS = DW + 2;                 // queued: v per dim, row/unsure, column
  constexpr int QN = 32 / G;                 // queue entries per warp
  extern __shared__ float ap_smem[];
  const int w = ix.w, D = ix.D;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int g = threadIdx.x % G;
  const int f0 = 16 * g;                     // this lane's first dim
  const int64_t a0 = int64_t(blockIdx.x) * kSeg;
  const int64_t dlo = int64_t(ix.excl) + 1 + (ybase + int64_t(blockIdx.y)) * NDG;
  if (dlo >= ix.M || a0 >= ix.M - dlo) return;                  // block-uniform
  const int64_t delta = dlo + threadIdx.x / G;
  const bool live = delta < ix.M && a0 < ix.M - delta;
  const int64_t a1 = live ? min(a0 + kSeg, ix.M - delta) : a0;
  const int64_t nrow = min(int64_t(kSeg), ix.M - dlo - a0);
  float* nuo = ap_smem;                                         // [RS][DW] -(x_{a-1} - c_a)
  float* uin = nuo + RS * DW;                                   // [RS][DW] x_{a+w-1} - c_a
  float* rowc = uin + RS * DW;                                  // [RS][DW2] {-(mu_a - c_a) x2, w sigma_a x2}
  float* cav = rowc + RS * 2 * DW;                              // [2][DW]
  float* sprev = cav + 2 * DW;                                  // [DW]
  float* qall = sprev + DW;                                     // [warps][QN][QS]
  __shared__ int rflag[RS];
  const float wf = float(w);
  const double wd = double(w);
  const float2* nuo2 = reinterpret_cast<const float2*>(nuo);
  const float2* uin2 = reinterpret_cast<const float2*>(uin);
  const float4* rowc4 = reinterpret_cast<const float4*>(rowc);
  float2 qt[DH], s1b[DH], ncb[DH];
#pragma unroll
  for (int p = 0; p < DH; ++p) {
    const int fa = f0 + 2 * p, fb = fa + 1;
    qt[p] = make_float2(fa < D ? 0.f : -1.f, fb < D ? 0.f : -1.f);
    s1b[p] = make_float2(0.f, 0.f);
    ncb[p] = make_float2(live && fa < D ? -ix.mu_hi[int64_t(fa) * ix.M + a0 + delta] : 0.f,
                         live && fb < D ? -ix.mu_hi[int64_t(fb) * ix.M + a0 + delta] : 0.f);
  }
  const float t1 = thr / float(d), t2 = d >= 2 ? thr / float(d - 1) : thr;
  const float c1 = 1.f - t1 * t1 / (2.f * wf), c2 = 1.f - t2 * t2 / (2.f * wf);
  const float cd = 1.f - thr * thr / (2.f * wf);
  const float2 nc1 = make_float2(-c1, -c1), nc2 = make_float2(-c2, -c2), ncd = make_float2(-cd, -cd);
  const int need2 = d >= 2 ? 2 : 1;
  float* qst = qall + warp * QN * QS;
  int64_t aS = a0;
  auto drain = [&](int count) {
    __syncwarp();
    if (lane < count) {
      const float* st = qst + lane * QS;
      const uint32_t meta = __float_as_uint(st[DW]);
      const int r = int(meta >> 1);
      const bool uns = (meta & 1u) != 0;
      float dist[DW];
#pragma unroll
      for (int f = 0; f < DW; ++f) {
        dist[f] = INFINITY;
        if (f < D) {
          const float wsa = rowc[(r * DW2 + (f >> 1)) * 4 + 2 + (f & 1)];
          const float corr = st[f] / wsa;
          dist[f] = sqrtf(fmaxf(2.f * wf * (1.f - corr), 0.f));
        }
      }
      const float sm = uns ? 0.f : sum_d_smallest<DW>(dist, D, d);
      if (sm <= thr && sm > rc.lo) record_pair(rc, aS + r, int64_t(__float_as_uint(st[DW + 1])), sm);
    }
    __syncwarp();
  };
  int qn = 0;                       // queued diagonals of this warp (warp-uniform)
  for (int stage = 0; aS < a0 + nrow; ++stage, aS += RS) {
    const int nsub = int(min(int64_t(RS), a0 + nrow - aS));
    float* cnew = cav + (stage & 1) * DW;
    const float* cold = cav + ((stage & 1) ^ 1) * DW;
    __syncthreads();                // the previous stage is fully consumed
    if (threadIdx.x < DW) {
      const int f = threadIdx.x;
      const float c = f < D ? ix.mu_hi[int64_t(f) * ix.M + aS] : 0.f;
      cnew[f] = c;
      sprev[f] = (f < D && aS >= 1) ? float(wd * (ix.mu[int64_t(f) * ix.M + aS - 1] - double(c))) : 0.f;
    }
    for (int r = threadIdx.x; r < RS; r += blockDim.x) rflag[r] = 0;
    __syncthreads();
    for (int q = threadIdx.x; q < nsub * DW; q += blockDim.x) {
      const int r = q / DW, f = q - r * DW;
      const int64_t a = aS + r;
      float* rcq = rowc + (r * DW2 + (f >> 1)) * 4 + (f & 1);
      if (f < D) {
        const float c = cnew[f];
        nuo[q] = a >= 1 ? c - X[(a - 1) * DW + f] : 0.f;
        uin[q] = X[(a + w - 1) * DW + f] - c;
        const double m = ix.mu[int64_t(f) * ix.M + a], sg = ix.sig[int64_t(f) * ix.M + a];
        const double dm = m - double(c), v = sg * sg;
        const bool ok = v > 1e-4 * (v + dm * dm) && ix.inv_sig[int64_t(f) * ix.M + a] != 0.f;
        rcq[0] = ok ? float(-dm) : 0.f;
        rcq[2] = ok ? float(wd * sg) : 1.f;
        if (!ok) atomicOr(&rflag[r], 1);
      } else {
        nuo[q] = uin[q] = 0.f;
        rcq[0] = 0.f;
        rcq[2] = 0.f;
      }
    }
    __syncthreads();
    if (stage == 0) {
      for (int t = 0; t < (live ? w : 0); ++t) {
        float xa[16], xb[16];
        load_row<16>(X + f0, (a0 + t) * G, xa);                 // same address over the block
        load_row<16>(X + f0, (a0 + delta + t) * G, xb);
#pragma unroll
        for (int p = 0; p < DH; ++p) {
          const float2 u = make_float2(xa[2 * p] - cnew[f0 + 2 * p], xa[2 * p + 1] - cnew[f0 + 2 * p + 1]);
          const float2 v = __fadd2_rn(make_float2(xb[2 * p], xb[2 * p + 1]), ncb[p]);
          qt[p] = __ffma2_rn(u, v, qt[p]);
          s1b[p] = __fadd2_rn(s1b[p], v);
        }
      }
    } else if (aS - 1 < a1) {
#pragma unroll
      for (int p = 0; p < DH; ++p) {
        const int fa = f0 + 2 * p, fb = fa + 1;
        const float2 dr = make_float2(cold[fa] - cnew[fa], cold[fb] - cnew[fb]);
        qt[p] = __ffma2_rn(dr, s1b[p], qt[p]);
        const float2 cbn = make_float2(fa < D ? ix.mu_hi[int64_t(fa) * ix.M + aS - 1 + delta] : 0.f,
                                       fb < D ? ix.mu_hi[int64_t(fb) * ix.M + aS - 1 + delta] : 0.f);
        const float2 dc = make_float2(cbn.x + ncb[p].x, cbn.y + ncb[p].y);
        qt[p] = __ffma2_rn(make_float2(-dc.x, -dc.y), make_float2(sprev[fa], sprev[fb]), qt[p]);
        s1b[p] = __ffma2_rn(make_float2(-wf, -wf), dc, s1b[p]);
        ncb[p] = make_float2(-cbn.x, -cbn.y);
      }
    }
    for (int r = 0; r < nsub; ++r) {
      const int64_t a = aS + r;
      const int64_t b = a + delta;
      const bool act = a < a1;
      float isb[16];
      int unsure = rflag[r];
      if (act) {
        if (r > 0 || stage > 0) {
          float ob[16], ib[16];
          load_row_v8<16>(X + f0, (b - 1) * G, ob);
          load_row_v8<16>(X + f0, (b + w - 1) * G, ib);
#pragma unroll
          for (int p = 0; p < DH; ++p) {
            const float2 o = make_float2(ob[2 * p], ob[2 * p + 1]);
            const float2 i = make_float2(ib[2 * p], ib[2 * p + 1]);
            const float2 vo = __fadd2_rn(o, ncb[p]), vi = __fadd2_rn(i, ncb[p]);
            qt[p] = __ffma2_rn(uin2[r * DW2 + f0 / 2 + p], vi, __ffma2_rn(nuo2[r * DW2 + f0 / 2 + p], vo, qt[p]));
            s1b[p] = __ffma2_rn(make_float2(-1.f, -1.f), o, __fadd2_rn(s1b[p], i));
          }
        }
        load_row_v8<16>(ix.isW + f0, b * G, isb);
        unsure |= ix.cflag[b];
      } else {
#pragma unroll
        for (int f = 0; f < 16; ++f) isb[f] = 0.f;
      }
      uint32_t all1 = 0xffffffffu;
      int negs = 0;                 // dims failing x(d)'s test (low half) and x(2)'s (high half)
      float2 v[DH];
#pragma unroll
      for (int p = 0; p < DH; ++p) {
        const float4 rq = rowc4[r * DW2 + f0 / 2 + p];
        const float2 u = __ffma2_rn(make_float2(rq.x, rq.y), s1b[p], qt[p]);
        v[p] = __fmul2_rn(u, make_float2(isb[2 * p], isb[2 * p + 1]));
        const float2 wsa = make_float2(rq.z, rq.w);
        const float2 e1 = __ffma2_rn(nc1, wsa, v[p]);
        const float2 ed = __ffma2_rn(ncd, wsa, v[p]);
        const float2 e2 = __ffma2_rn(nc2, wsa, v[p]);
        all1 &= __float_as_uint(e1.x) & __float_as_uint(e1.y);
        negs += int(__float_as_uint(ed.x) >> 31) + int(__float_as_uint(ed.y) >> 31) +
                ((int(__float_as_uint(e2.x) >> 31) + int(__float_as_uint(e2.y) >> 31)) << 16);
      }
      // the diagonal's totals over its G lanes
#pragma unroll
      for (int o = 1; o < G; o <<= 1) {
        all1 &= __shfl_xor_sync(0xffffffffu, all1, o);
        negs += __shfl_xor_sync(0xffffffffu, negs, o);
        unsure |= __shfl_xor_sync(0xffffffffu, unsure, o);
      }
      const int negd = negs & 0xffff, neg2 = negs >> 16;
      const bool cand = act && (unsure || ((all1 >> 31) == 0u && DW - negd >= d && DW - neg2 >= need2));
      const unsigned m = __ballot_sync(0xffffffffu, cand);
      if (!m) continue;
      const int n = __popc(m) / G;                  // candidate diagonals of this step
      if (qn + n > QN) {
        drain(qn);
        qn = 0;
      }
      if (cand) {
        const int base = lane - g;                  // the diagonal's first lane
        const int pos = qn + __popc(m & ((1u << base) - 1u)) / G;
        float* st = qst + pos * QS;
#pragma unroll
        for (int p = 0; p < DH; ++p) {
          st[f0 + 2 * p] = v[p].x;
          st[f0 + 2 * p + 1] = v[p].y;
        }
        if (g == 0) {
          st[DW] = __uint_as_float((uint32_t(r) << 1) | (unsure ? 1u : 0u));
          st[DW + 1] = __uint_as_float(uint32_t(b));
        }
      }
      qn += n;
      if (qn == QN) {
        drain(QN);
        qn = 0;
      }
    }
    drain(qn);                      // queued diagonals refer to this stage's rows
    qn = 0;
  }
}

// Wide series (D > 16): per-window means and 1/sigma are read per step;
// every thread of a block walks the same row windows a (their values are
// broadcast loads) against its own diagonal.  Only the D centred cross
// products live in registers: the row centring (the block's first row
// window mean) and each thread's column centring sit in shared memory, and
// a pair's squared distances are computed twice, the second time only for
// a pair that has at least d dims within the threshold (the square roots
// and the sum of the d smallest).
template <int DM, bool ROWMIN>
__global__ void __launch_bounds__(kDiagBlock, DM <= 32 ? 3 : 2)
k_allpairs_wide(Index ix, int d, float thr, ApRec rc, float* __restrict__ rowmin, int64_t ybase) {
  extern __shared__ float wd_smem[];
  float* s_ca = wd_smem;                         // [DM]
  float* s_cb = wd_smem + DM;                    // [DM][kDiagBlock]
  const int64_t delta = int64_t(ix.excl) + 1 + (ybase + int64_t(blockIdx.y)) * kDiagBlock + threadIdx.x;
  const int64_t a0 = int64_t(blockIdx.x) * kSeg;
  const int D = ix.D, w = ix.w;
  if (threadIdx.x < DM) s_ca[threadIdx.x] = int(threadIdx.x) < D ? ix.mu_hi[int64_t(threadIdx.x) * ix.M + a0] : 0.f;
  __syncthreads();
  if (delta >= ix.M || a0 >= ix.M - delta) return;
  const int64_t a1 = min(a0 + kSeg, ix.M - delta);
  const float wf = float(w);
  const float thr2 = thr * thr * (1.f + 1e-6f);      // a rounding of slack on the square
  float* cb = s_cb + threadIdx.x;                    // cb[f * kDiagBlock]
  float qt[DM];
  // direct start: centred dot products of windows a0 and a0 + delta
#pragma unroll
  for (int f = 0; f < DM; ++f) {
    qt[f] = 0.f;
    if (f < D) {
      const float* xh = ix.xs_hi + int64_t(f) * ix.n;
      const float* xl = ix.has_lo ? ix.xs_lo + int64_t(f) * ix.n : nullptr;
      const float ca = s_ca[f], cbf = ix.mu_hi[int64_t(f) * ix.M + a0 + delta];
      cb[f * kDiagBlock] = cbf;
      float acc = 0.f;
      for (int t = 0; t < w; ++t)
        acc = fmaf(xv(xh, xl, a0 + t) - ca, xv(xh, xl, a0 + delta + t) - cbf, acc);
      qt[f] = acc;
    }
  }
  // squared z-normalised distance of dim f for the current (a, b)
  auto sq_of = [&](int f, int64_t a, int64_t b) {
    const int64_t oa = int64_t(f) * ix.M + a, ob = int64_t(f) * ix.M + b;
    const float isa = ix.inv_sig[oa], isb = ix.inv_sig[ob];
    const float da = ix.mu_hi[oa] - s_ca[f], db = ix.mu_hi[ob] - cb[f * kDiagBlock];
    const float cov = qt[f] / wf - da * db;
    const float na = isa > 0.f ? wf : 0.f, nb = isb > 0.f ? wf : 0.f;
    return fmaxf(na + nb - 2.f * wf * cov * isa * isb, 0.f);
  };
  for (int64_t a = a0; a < a1; ++a) {
    const int64_t b = a + delta;
    if (a > a0) {
#pragma unroll
      for (int f = 0; f < DM; ++f) {
        if (f < D) {
          const float* xh = ix.xs_hi + int64_t(f) * ix.n;
          const float* xl = ix.has_lo ? ix.xs_lo + int64_t(f) * ix.n : nullptr;
          const float ca = s_ca[f], cbf = cb[f * kDiagBlock];
          const float out_a = xv(xh, xl, a - 1) - ca, out_b = xv(xh, xl, b - 1) - cbf;
          const float in_a = xv(xh, xl, a + w - 1) - ca, in_b = xv(xh, xl, b + w - 1) - cbf;
          qt[f] = fmaf(in_a, in_b, fmaf(-out_a, out_b, qt[f]));
        }
      }
    }
    int near = 0;
#pragma unroll
    for (int f = 0; f < DM; ++f)
      if (f < D) near += sq_of(f, a, b) <= thr2;
    if (ROWMIN || near >= d) {
      float dist[DM];
#pragma unroll
      for (int f = 0; f < DM; ++f) dist[f] = f < D ? sqrtf(sq_of(f, a, b)) : INFINITY;
      const float sm = sum_d_smallest<DM>(dist, D, d);
      if (ROWMIN) {
        atomicMin(reinterpret_cast<int*>(rowmin + a), __float_as_int(sm));
        atomicMin(reinterpret_cast<int*>(rowmin + b), __float_as_int(sm));
      } else if (sm <= thr && sm > rc.lo) {
        record_pair(rc, a, b, sm);
      }
    }
  }
}

// the row kernel stages kRowSub+w points of every dimension in shared
// memory, the row sums, and a queue of 32 candidate pairs per warp
size_t rows_smem(int w, int dp) {
  return (size_t((kRowSub + w) * dp + 2 * kRowSub * dp + 3 * dp) +
          size_t(kDiagBlock) * (3 * dp + 2) + 2 * size_t(kDiagBlock)) * sizeof(float);
}

bool rows_fit(int w, int dp) { return rows_smem(w, dp) <= size_t(200) * 1024; }

// the wide row kernel: two staged points and two row sums per row and dim
// for kRowSub2 rows of DW dims, a queue of 32/G diagonals per warp
size_t rows2_smem(int w, int dw) {
  (void)w;                                   // staging does not grow with w
  const int G = dw / 16, QN = 32 / G;
  return (size_t(4 * kRowSub2 * dw + 3 * dw) +
          size_t(kDiagBlock / 32) * QN * (3 * dw + 2) + 2 * size_t(kDiagBlock / 32) * QN) * sizeof(float);
}

// the statistics sweep: two staged points and the row factors per row and
// dim for rs rows, a queue of 32 candidates (v per dim, row, column) per warp
size_t rows3_smem(int dp, int rs) {
  return size_t(4 * rs * dp + 3 * dp + kDiagBlock * (dp + 2)) * sizeof(float);
}

// the wide statistics sweep: rows3's staging for kRowSub2 rows of DW dims,
// a queue of 32/G diagonals per warp
size_t rows4_smem(int dw) {
  const int G = dw / 16, QN = 32 / G;
  return size_t(4 * kRowSub2 * dw + 3 * dw + (kDiagBlock / 32) * QN * (dw + 2)) * sizeof(float);
}

// ---- recording-sweep variants and their autotuner -------------------------
// A float32 index has several forms of the recording sweep, all recording
// the same pairs: for D <= 16 the statistics form with two stage heights
// and the slid form (k_allpairs_rows, whose staging grows with w); for
// 16 < D <= 64 the statistics and the slid wide forms.  Which one is
// fastest depends on the padded D, w and M.  The grid of every launch
// below may be cut to its first gy_max diagonal blocks (the autotuner's
// probe).

template <int DP, int RS, int MINB>
cudaError_t rows3_launch(const Index& ix, int d, float thr, const ApRec& rc, cudaStream_t s,
                         int64_t gy_max) {
  const int64_t ndiag = ix.M - (ix.excl + 1);
  const int64_t gy = std::min<int64_t>((ndiag + kDiagBlock - 1) / kDiagBlock, gy_max);
  const size_t smem = rows3_smem(DP, RS);
  cudaError_t e = allow_smem(reinterpret_cast<const void*>(k_allpairs_rows3<DP, RS, MINB>), smem);
  if (e != cudaSuccess) return e;
  for (int64_t y0 = 0; y0 < gy; y0 += 65535) {
    dim3 grid{unsigned((ix.M + kSeg - 1) / kSeg), unsigned(std::min<int64_t>(65535, gy - y0)), 1u};
    MOMENTI_LAUNCH("allpairs", s, k_allpairs_rows3<DP, RS, MINB><<<grid, kDiagBlock, smem, s>>>(ix, d, thr, rc, y0));
  }
  return cudaGetLastError();
}

template <int DP>
cudaError_t rows_slid_launch(const Index& ix, int d, float thr, const ApRec& rc, cudaStream_t s,
                             int64_t gy_max) {
  const int64_t ndiag = ix.M - (ix.excl + 1);
  const int64_t gy = std::min<int64_t>((ndiag + kDiagBlock - 1) / kDiagBlock, gy_max);
  const size_t smem = rows_smem(ix.w, DP);
  cudaError_t e = allow_smem(reinterpret_cast<const void*>(k_allpairs_rows<DP, false>), smem);
  if (e != cudaSuccess) return e;
  for (int64_t y0 = 0; y0 < gy; y0 += 65535) {
    dim3 grid{unsigned((ix.M + kSeg - 1) / kSeg), unsigned(std::min<int64_t>(65535, gy - y0)), 1u};
    MOMENTI_LAUNCH("allpairs", s, k_allpairs_rows<DP, false><<<grid, kDiagBlock, smem, s>>>(ix, d, thr, rc, nullptr, y0));
  }
  return cudaGetLastError();
}

template <int DW>
cudaError_t rows4_launch(const Index& ix, int d, float thr, const ApRec& rc, cudaStream_t s,
                         int64_t gy_max) {
  const int64_t ndiag = ix.M - (ix.excl + 1);
  constexpr int NDG = kDiagBlock / (DW / 16);
  const int64_t gy = std::min<int64_t>((ndiag + NDG - 1) / NDG, gy_max);
  const size_t smem = rows4_smem(DW);
  cudaError_t e = allow_smem(reinterpret_cast<const void*>(k_allpairs_rows4<DW>), smem);
  if (e != cudaSuccess) return e;
  for (int64_t y0 = 0; y0 < gy; y0 += 65535) {
    dim3 grid{unsigned((ix.M + kSeg - 1) / kSeg), unsigned(std::min<int64_t>(65535, gy - y0)), 1u};
    MOMENTI_LAUNCH("allpairs", s, k_allpairs_rows4<DW><<<grid, kDiagBlock, smem, s>>>(ix, ix.xW, d, thr, rc, y0));
  }
  return cudaGetLastError();
}

template <int DW>
cudaError_t rows2_launch(const Index& ix, int d, float thr, const ApRec& rc, cudaStream_t s,
                         int64_t gy_max) {
  const int64_t ndiag = ix.M - (ix.excl + 1);
  constexpr int NDG = kDiagBlock / (DW / 16);
  const int64_t gy = std::min<int64_t>((ndiag + NDG - 1) / NDG, gy_max);
  const size_t smem = rows2_smem(ix.w, DW);
  cudaError_t e = allow_smem(reinterpret_cast<const void*>(k_allpairs_rows2<DW, false>), smem);
  if (e != cudaSuccess) return e;
  for (int64_t y0 = 0; y0 < gy; y0 += 65535) {
    dim3 grid{unsigned((ix.M + kSeg - 1) / kSeg), unsigned(std::min<int64_t>(65535, gy - y0)), 1u};
    MOMENTI_LAUNCH("allpairs", s, k_allpairs_rows2<DW, false><<<grid, kDiagBlock, smem, s>>>(ix, ix.xW, d, thr, rc, nullptr, y0));
  }
  return cudaGetLastError();
}

template <int DW, bool ROWMIN>
cudaError_t rows2_dispatch(const Index& ix, int d, float thr, const ApRec& rc, float* rowmin,
                           cudaStream_t s) {
  const int64_t ndiag = ix.M - (ix.excl + 1);
  constexpr int NDG = kDiagBlock / (DW / 16);
  const int64_t gy = (ndiag + NDG - 1) / NDG;
  const size_t smem = rows2_smem(ix.w, DW);
  cudaError_t e = allow_smem(reinterpret_cast<const void*>(k_allpairs_rows2<DW, ROWMIN>), smem);
  if (e != cudaSuccess) return e;
  for (int64_t y0 = 0; y0 < gy; y0 += 65535) {
    dim3 grid{unsigned((ix.M + kSeg - 1) / kSeg), unsigned(std::min<int64_t>(65535, gy - y0)), 1u};
    MOMENTI_LAUNCH("allpairs", s, k_allpairs_rows2<DW, ROWMIN><<<grid, kDiagBlock, smem, s>>>(ix, ix.xW, d, thr, rc, rowmin, y0));
  }
  return cudaGetLastError();
}

}  // namespace

}  // namespace momenti
