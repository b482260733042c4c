// Candidate verification (Algorithm 1, line 15) and the exact all-pairs
// path (Algorithm 1, line 20).
//
// Per pair: the z-normalised Euclidean distance of Eq. (zned) in every
// dimension, computed directly from the centred windows,
//   dist_f^2 = sum_t ((x_a[t] - mu_a) / sigma_a - (x_b[t] - mu_b) / sigma_b)^2,
// then dist_d = the sum of the d smallest (Definition distdims, ties to the
// lower dimension), dims_d as a mask and dist_d^max (Eq. distdmax).  One
// warp per pair, lanes over t, in float32 (the traversal) or float64 (the
// final re-verification).
//
// The all-pairs path walks the diagonals b - a = delta of the distance
// matrix: along a diagonal the dot product of the two centred windows
// slides by one product in and one out, restarted from a direct sum every
// kSeg steps; the per-dimension distance follows from the Pearson form
// dist^2 = n_a + n_b - 2 w corr (Section 2), n = w for non-flat windows and
// 0 for flat ones.  Pairs whose dist_d may be <= tau are collected and then
// verified exactly by the direct form above.
#include "internal.h"

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

// One warp per candidate event: distances; a pair with dist_d < tau is
// recorded (with its repetition) and offered to the set of close pairs.
__global__ void __launch_bounds__(256)
k_verify_events(Index ix, int d, HashSet hs, const Event* __restrict__ ev,
                unsigned long long* __restrict__ counters, uint64_t ev_cap, float tau,
                PairRec* __restrict__ rec, uint64_t rec_cap) {
  const int lane = threadIdx.x & 31;
  uint64_t cnt = counters[0];
  if (cnt > ev_cap) cnt = ev_cap;
  const uint64_t nw = uint64_t(gridDim.x) * (blockDim.x >> 5);
  for (uint64_t q = (blockIdx.x * uint64_t(blockDim.x) + threadIdx.x) >> 5; q < cnt; q += nw) {
    const Event e = ev[q];
    float dist[2];
    pair_distances<float>(ix, e.a, e.b, dist);
    VerifyOut v = select_d<float>(dist, ix.D, d);
    if (lane != 0) continue;
    if (!(float(v.dist_d) < tau)) {
      atomicAdd(&counters[3], 1ull);
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

constexpr int kSeg = 64;        // diagonal steps between direct restarts
constexpr int kDiagBlock = 128; // diagonals per CTA

__device__ __forceinline__ float xv(const float* xh, const float* xl, int64_t t) {
  return xl ? xh[t] + xl[t] : xh[t];
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

template <int DM, bool ROWMIN>
__global__ void __launch_bounds__(kDiagBlock)
k_allpairs(Index ix, int d, float tau, uint64_t* __restrict__ out, uint64_t cap,
           unsigned long long* __restrict__ count, float* __restrict__ rowmin) {
  const int64_t delta = int64_t(ix.excl) + 1 + int64_t(blockIdx.y) * kDiagBlock + threadIdx.x;
  const int64_t a0 = int64_t(blockIdx.x) * kSeg;
  if (delta >= ix.M || a0 >= ix.M - delta) return;
  const int64_t a1 = min(a0 + kSeg, ix.M - delta);
  const int D = ix.D, w = ix.w;
  const float wf = float(w);
  float qt[DM], ca[DM], cb[DM];
  // direct start: centred dot products of windows a0 and a0 + delta
#pragma unroll
  for (int f = 0; f < DM; ++f) {
    qt[f] = 0.f; ca[f] = 0.f; cb[f] = 0.f;
    if (f < D) {
      const float* xh = ix.xs_hi + int64_t(f) * ix.n;
      const float* xl = ix.has_lo ? ix.xs_lo + int64_t(f) * ix.n : nullptr;
      ca[f] = ix.mu_hi[int64_t(f) * ix.M + a0];
      cb[f] = ix.mu_hi[int64_t(f) * ix.M + a0 + delta];
      float s = 0.f;
      for (int t = 0; t < w; ++t)
        s = fmaf(xv(xh, xl, a0 + t) - ca[f], xv(xh, xl, a0 + delta + t) - cb[f], s);
      qt[f] = s;
    }
  }
  const float thr = tau * 1.01f + 1e-2f;
  for (int64_t a = a0; a < a1; ++a) {
    const int64_t b = a + delta;
    if (a > a0) {
#pragma unroll
      for (int f = 0; f < DM; ++f) {
        if (f < D) {
          const float* xh = ix.xs_hi + int64_t(f) * ix.n;
          const float* xl = ix.has_lo ? ix.xs_lo + int64_t(f) * ix.n : nullptr;
          float out_a = xv(xh, xl, a - 1) - ca[f], out_b = xv(xh, xl, b - 1) - cb[f];
          float in_a = xv(xh, xl, a + w - 1) - ca[f], in_b = xv(xh, xl, b + w - 1) - cb[f];
          qt[f] = fmaf(in_a, in_b, fmaf(-out_a, out_b, qt[f]));
        }
      }
    }
    float dist[DM];
    int near = 0;
#pragma unroll
    for (int f = 0; f < DM; ++f) {
      dist[f] = INFINITY;
      if (f < D) {
        const int64_t oa = int64_t(f) * ix.M + a, ob = int64_t(f) * ix.M + b;
        const float isa = ix.inv_sig[oa], isb = ix.inv_sig[ob];
        const float da = ix.mu_hi[oa] - ca[f], db = ix.mu_hi[ob] - cb[f];
        const float cov = qt[f] / wf - da * db;
        const float na = isa > 0.f ? wf : 0.f, nb = isb > 0.f ? wf : 0.f;
        const float sq = na + nb - 2.f * wf * cov * isa * isb;
        dist[f] = sqrtf(fmaxf(sq, 0.f));
        near += dist[f] <= thr;
      }
    }
    if (ROWMIN) {
      float s = sum_d_smallest<DM>(dist, D, d);
      atomicMin(reinterpret_cast<int*>(rowmin + a), __float_as_int(s));
      atomicMin(reinterpret_cast<int*>(rowmin + b), __float_as_int(s));
    } else if (near >= d) {
      float s = sum_d_smallest<DM>(dist, D, d);
      if (s <= thr) {
        unsigned long long pos = atomicAdd(count, 1ull);
        if (pos < cap) out[pos] = (uint64_t(a) << 32) | uint64_t(b);
      }
    }
  }
}

template <bool ROWMIN>
cudaError_t allpairs_dispatch(const Index& ix, int d, float tau, uint64_t* out, uint64_t cap,
                              unsigned long long* count, float* rowmin, cudaStream_t s) {
  const int64_t ndiag = ix.M - (ix.excl + 1);
  if (ndiag <= 0) return cudaSuccess;
  dim3 grid{unsigned((ix.M + kSeg - 1) / kSeg), unsigned((ndiag + kDiagBlock - 1) / kDiagBlock), 1u};
  if (ix.D <= 4)
    MOMENTI_LAUNCH("allpairs", s, k_allpairs<4, ROWMIN><<<grid, kDiagBlock, 0, s>>>(ix, d, tau, out, cap, count, rowmin));
  else if (ix.D <= 8)
    MOMENTI_LAUNCH("allpairs", s, k_allpairs<8, ROWMIN><<<grid, kDiagBlock, 0, s>>>(ix, d, tau, out, cap, count, rowmin));
  else if (ix.D <= 16)
    MOMENTI_LAUNCH("allpairs", s, k_allpairs<16, ROWMIN><<<grid, kDiagBlock, 0, s>>>(ix, d, tau, out, cap, count, rowmin));
  else if (ix.D <= 32)
    MOMENTI_LAUNCH("allpairs", s, k_allpairs<32, ROWMIN><<<grid, kDiagBlock, 0, s>>>(ix, d, tau, out, cap, count, rowmin));
  else
    MOMENTI_LAUNCH("allpairs", s, k_allpairs<64, ROWMIN><<<grid, kDiagBlock, 0, s>>>(ix, d, tau, out, cap, count, rowmin));
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_verify_events(const Index& ix, int d, const HashSet& hs,
                                 const CollideScratch& cs, float tau, PairRec* rec,
                                 uint64_t rec_cap, cudaStream_t s) {
  MOMENTI_LAUNCH("verify_events", s, k_verify_events<<<152 * 8, 256, 0, s>>>(ix, d, hs, cs.events, cs.counters, cs.ev_cap, tau, rec, rec_cap));
  return cudaGetLastError();
}

cudaError_t launch_verify_pairs(const Index& ix, int d, const uint64_t* pairs, int64_t m,
                                int fp64, double* per_dim, double* dist_d, uint64_t* dims,
                                cudaStream_t s) {
  if (m <= 0) return cudaSuccess;
  int64_t g = (m + 7) / 8;
  if (g > 152 * 16) g = 152 * 16;
  MOMENTI_LAUNCH("verify_pairs", s, k_verify_pairs<<<unsigned(g), 256, 0, s>>>(ix, d, pairs, m, fp64, per_dim, dist_d, dims));
  return cudaGetLastError();
}

cudaError_t launch_allpairs(const Index& ix, int d, float tau, uint64_t* out, uint64_t cap,
                            unsigned long long* count, cudaStream_t s) {
  return allpairs_dispatch<false>(ix, d, tau, out, cap, count, nullptr, s);
}

cudaError_t launch_allpairs_rowmin(const Index& ix, int d, float* rowmin, cudaStream_t s) {
  return allpairs_dispatch<true>(ix, d, 0.f, nullptr, 0, nullptr, rowmin, s);
}

}  // namespace momenti
