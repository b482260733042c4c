// Candidate verification (the distance check of Algorithm 1's inner loop)
// and the exact all-pairs path (the final fallback of Algorithm 1).
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

#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <map>
#include <mutex>
#include <string>
#include <tuple>
#include <vector>

#include "k_verify_kernels.cuh"

namespace momenti {

namespace {

bool aligned32(const void* q) { return (reinterpret_cast<uintptr_t>(q) & 31u) == 0; }

// Candidates for this index (0 when the recording sweep has no variants:
// float64 input, no point-major copy).  The statistics forms read column
// rows with 256-bit loads, so their rows must start on 32-byte boundaries
// (the pool aligns far beyond that; checked, not assumed).
int sweep_variants(const Index& ix) {
  if (ix.xW && ix.isW && rows2_usable(ix) && aligned32(ix.xW) && aligned32(ix.isW)) return 2;
  if (ix.isT && ix.xT && !ix.has_lo && aligned32(ix.xT) && aligned32(ix.isT))
    return rows_fit(ix.w, ix.Dp) ? 3 : 2;
  return 0;
}

// Variant v: wide: 0 statistics, 1 slid; D <= 16: 0 statistics with the
// taller stage, 1 statistics with half of it, 2 slid.
cudaError_t sweep_launch(const Index& ix, int v, int d, float thr, const ApRec& rc, cudaStream_t s,
                         int64_t gy_max) {
  if (ix.xW) {
    if (ix.DW == 32) return v == 0 ? rows4_launch<32>(ix, d, thr, rc, s, gy_max) : rows2_launch<32>(ix, d, thr, rc, s, gy_max);
    return v == 0 ? launch_rows4_64(ix, d, thr, rc, s, gy_max) : launch_rows2_64(ix, d, thr, rc, s, gy_max);
  }
  switch (ix.Dp) {
    case 4:
      if (v == 0) return rows3_launch<4, kRowSub3, 3>(ix, d, thr, rc, s, gy_max);
      if (v == 1) return rows3_launch<4, kRowSub3 / 2, 3>(ix, d, thr, rc, s, gy_max);
      return rows_slid_launch<4>(ix, d, thr, rc, s, gy_max);
    case 8:
      if (v == 0) return rows3_launch<8, kRowSub3, 3>(ix, d, thr, rc, s, gy_max);
      if (v == 1) return rows3_launch<8, kRowSub3 / 2, 3>(ix, d, thr, rc, s, gy_max);
      return rows_slid_launch<8>(ix, d, thr, rc, s, gy_max);
    default:
      if (v == 0) return rows3_launch<16, kRowSub3 / 2, 2>(ix, d, thr, rc, s, gy_max);
      if (v == 1) return rows3_launch<16, kRowSub3 / 4, 2>(ix, d, thr, rc, s, gy_max);
      return rows_slid_launch<16>(ix, d, thr, rc, s, gy_max);
  }
}

struct TuneKey {
  int dev, dp, lw, lm;
  bool operator<(const TuneKey& o) const {
    return std::tie(dev, dp, lw, lm) < std::tie(o.dev, o.dp, o.lw, o.lm);
  }
};
std::mutex& tune_mu() {
  static std::mutex m;
  return m;
}
std::map<TuneKey, int>& tune_map() {
  static std::map<TuneKey, int> t;
  return t;
}
int ilog2(int64_t x) {
  int l = 0;
  while (x > 1) { x >>= 1; ++l; }
  return l;
}

// The variant the sweep of this index runs: MOMENTI_SWEEP_VARIANT=v forces
// one; MOMENTI_AUTOTUNE=0 takes variant 0; otherwise the cached choice for
// (device, padded D, log2 w, log2 M), or, the first time, the fastest
// candidate on a probe: every candidate runs three times over the grid's
// first diagonal blocks (about four waves of CTAs, the longest diagonals)
// with a negative threshold, which records nothing; the faster of the last
// two runs counts (CUDA events on the sweep's stream).  Probes run one at a
// time in the process.
int sweep_variant(const Index& ix, int d, const ApRec& rc, cudaStream_t s) {
  const int nv = sweep_variants(ix);
  if (const char* f = std::getenv("MOMENTI_SWEEP_VARIANT"); f && f[0] >= '0' && f[0] <= '9')
    return std::min(nv - 1, int(f[0] - '0'));
  if (nv <= 1) return 0;
  if (const char* e = std::getenv("MOMENTI_AUTOTUNE"); e && e[0] == '0') return 0;
  int dev = 0;
  cudaGetDevice(&dev);
  const TuneKey key{dev, ix.xW ? ix.DW : ix.Dp, ilog2(ix.w), ilog2(ix.M)};
  {
    std::lock_guard<std::mutex> g(tune_mu());
    auto it = tune_map().find(key);
    if (it != tune_map().end()) return it->second;
  }
  // one probe at a time in the process (probes of other threads would
  // share the GPU with this one and distort its timings)
  static std::mutex probe_mu;
  std::lock_guard<std::mutex> probe_lock(probe_mu);
  {
    std::lock_guard<std::mutex> g(tune_mu());
    auto it = tune_map().find(key);
    if (it != tune_map().end()) return it->second;
  }
  const int64_t nbx = (ix.M + kSeg - 1) / kSeg;
  const int64_t gy_probe = std::max<int64_t>(1, (int64_t(sm_count()) * 8 + nbx - 1) / nbx);
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    if (e0) cudaEventDestroy(e0);
    return 0;
  }
  int best = 0;
  float best_ms = INFINITY;
  std::string line;
  for (int v = 0; v < nv; ++v) {
    float ms = INFINITY;
    bool ok = true;
    for (int rep = 0; rep < 3 && ok; ++rep) {    // a warm-up, then the faster of two
      float t = INFINITY;
      ok = cudaEventRecord(e0, s) == cudaSuccess &&
           sweep_launch(ix, v, d, -1.f, rc, s, gy_probe) == cudaSuccess &&
           cudaEventRecord(e1, s) == cudaSuccess && cudaEventSynchronize(e1) == cudaSuccess &&
           cudaEventElapsedTime(&t, e0, e1) == cudaSuccess;
      if (rep > 0) ms = std::min(ms, t);
    }
    if (!ok) {
      cudaGetLastError();       // a candidate that cannot launch is skipped
      continue;
    }
    line += " v" + std::to_string(v) + "=" + std::to_string(ms);
    if (ms < best_ms) {
      best_ms = ms;
      best = v;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  {
    std::lock_guard<std::mutex> g(tune_mu());
    tune_map().emplace(key, best);
  }
  if (const char* t = std::getenv("MOMENTI_TRACE"); t && t[0] == '1')
    std::fprintf(stderr, "momenti trace: sweep autotune dp=%d w=%d M=%lld ms:%s -> v%d\n", key.dp, ix.w,
                 (long long)ix.M, line.c_str(), best);
  return best;
}

// Column table of the statistics sweep: isT[b][f] = 1/sigma (0 for flat
// windows, 1 for padding dims) and cflag[b] = 1 when some dim of window b
// is flat or its column centring offset may be large against its sigma.
// The centring constant of a diagonal is the float32 mean of a column
// window b' in [b - kRowSub3, b] (the stage's first column), so b is marked
// when sigma^2 <= 1e-4 (sigma^2 + max |mean(b') - mean(b)|^2) there, the
// condition the rows kernels apply to the offset they actually carry.
__global__ void k_col_prep(Index ix) {
  const int64_t b = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (b >= ix.M) return;
  float* tab = ix.isT ? ix.isT : ix.isW;
  const int DP = ix.isT ? ix.Dp : ix.DW;
  int u = 0;
  for (int f = 0; f < DP; ++f) {
    float is = 1.f;
    if (f < ix.D) {
      const int64_t o = int64_t(f) * ix.M;
      is = ix.inv_sig[o + b];
      const float mb = ix.mu_hi[o + b];
      float dmax = 0.f;
      for (int64_t q = b > kRowSub3 ? b - kRowSub3 : 0; q <= b; ++q)
        dmax = fmaxf(dmax, fabsf(ix.mu_hi[o + q] - mb));
      const double sg = ix.sig[o + b], v = sg * sg, dm = double(dmax);
      u |= (is == 0.f) || !(v > 1e-4 * (v + dm * dm));
    }
    tab[b * DP + f] = is;
  }
  ix.cflag[b] = uint8_t(u);
}

}  // namespace

cudaError_t launch_col_prep(const Index& ix, cudaStream_t s) {
  if (!ix.isT && !ix.isW) return cudaSuccess;
  MOMENTI_LAUNCH("col_prep", s, k_col_prep<<<unsigned((ix.M + 255) / 256), 256, 0, s>>>(ix));
  return cudaGetLastError();
}

bool sweep_batchable(const Index& ix) {
  return !ix.xW && sweep_variants(ix) > 0;
}

cudaError_t launch_allpairs_batch(const std::vector<SweepJob>& jobs, cudaStream_t s) {
  if (jobs.empty()) return cudaSuccess;
  for (const auto& j : jobs)
    if (!sweep_batchable(j.ix)) return cudaErrorInvalidValue;
  // items of every job, largest series first; one persistent launch per
  // padded dimension count (the kernel's register and shared-memory shape)
  std::vector<int> order(jobs.size());
  for (size_t q = 0; q < jobs.size(); ++q) order[q] = int(q);
  std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return jobs[x].ix.M > jobs[y].ix.M; });
  SweepJob* djobs = nullptr;
  cudaError_t e = cudaMallocAsync(&djobs, jobs.size() * sizeof(SweepJob), s);
  if (e != cudaSuccess) return e;
  e = cudaMemcpyAsync(djobs, jobs.data(), jobs.size() * sizeof(SweepJob), cudaMemcpyHostToDevice, s);
  for (int dp : {4, 8, 16}) {
    std::vector<SweepItem> items;
    for (int q : order) {
      const Index& ix = jobs[q].ix;
      if (ix.Dp != dp || ix.M - (ix.excl + 1) <= 0) continue;
      const int64_t nbx = (ix.M + kSeg - 1) / kSeg;
      const int64_t gy = (ix.M - (ix.excl + 1) + kDiagBlock - 1) / kDiagBlock;
      for (int64_t by = 0; by < gy; ++by) {
        const int64_t dlo = int64_t(ix.excl) + 1 + by * kDiagBlock;
        for (int64_t bx = 0; bx < nbx && bx * kSeg < ix.M - dlo; ++bx)
          items.push_back(SweepItem{uint32_t(q), uint32_t(bx), uint32_t(by)});
      }
    }
    if (items.empty() || e != cudaSuccess) continue;
    SweepItem* ditems = nullptr;
    int* dnext = nullptr;
    if ((e = cudaMallocAsync(&ditems, items.size() * sizeof(SweepItem), s)) != cudaSuccess) break;
    if ((e = cudaMallocAsync(&dnext, sizeof(int), s)) != cudaSuccess) {
      cudaFreeAsync(ditems, s);
      break;
    }
    e = cudaMemcpyAsync(ditems, items.data(), items.size() * sizeof(SweepItem), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(dnext, 0, sizeof(int), s);
    const int per_sm = dp <= 8 ? 3 : 2;
    const int64_t grid = std::min<int64_t>(int64_t(sm_count()) * per_sm, int64_t(items.size()));
    const int nit = int(items.size());
    if (e == cudaSuccess) {
      if (dp == 4) {
        const size_t smem = rows3_smem(4, kRowSub3);
        e = allow_smem(reinterpret_cast<const void*>(k_allpairs_rows3_batch<4, kRowSub3, 3>), smem);
        if (e == cudaSuccess)
          MOMENTI_LAUNCH("allpairs_batch", s, k_allpairs_rows3_batch<4, kRowSub3, 3><<<unsigned(grid), kDiagBlock, smem, s>>>(djobs, ditems, nit, dnext));
      } else if (dp == 8) {
        const size_t smem = rows3_smem(8, kRowSub3);
        e = allow_smem(reinterpret_cast<const void*>(k_allpairs_rows3_batch<8, kRowSub3, 3>), smem);
        if (e == cudaSuccess)
          MOMENTI_LAUNCH("allpairs_batch", s, k_allpairs_rows3_batch<8, kRowSub3, 3><<<unsigned(grid), kDiagBlock, smem, s>>>(djobs, ditems, nit, dnext));
      } else {
        const size_t smem = rows3_smem(16, kRowSub3 / 2);
        e = allow_smem(reinterpret_cast<const void*>(k_allpairs_rows3_batch<16, kRowSub3 / 2, 2>), smem);
        if (e == cudaSuccess)
          MOMENTI_LAUNCH("allpairs_batch", s, k_allpairs_rows3_batch<16, kRowSub3 / 2, 2><<<unsigned(grid), kDiagBlock, smem, s>>>(djobs, ditems, nit, dnext));
      }
      if (e == cudaSuccess) e = cudaGetLastError();
    }
    cudaFreeAsync(ditems, s);
    cudaFreeAsync(dnext, s);
  }
  cudaFreeAsync(djobs, s);
  return e;
}

bool rows2_usable(const Index& ix) {
  return ix.xW && !ix.has_lo && (ix.DW == 32 || ix.DW == 64) &&
         rows2_smem(ix.w, ix.DW) <= size_t(220) * 1024;
}

namespace {


template <bool ROWMIN>
cudaError_t allpairs_dispatch(const Index& ix, int d, float thr, const ApRec& rc, float* rowmin,
                              cudaStream_t s) {
  const int64_t ndiag = ix.M - (ix.excl + 1);
  if (ndiag <= 0) return cudaSuccess;
  if constexpr (!ROWMIN) {
    if (sweep_variants(ix) > 0)
      return sweep_launch(ix, sweep_variant(ix, d, rc, s), d, thr, rc, s, int64_t(1) << 40);
  }
  if (rows2_usable(ix)) {
    if (ix.DW == 32) return rows2_dispatch<32, ROWMIN>(ix, d, thr, rc, rowmin, s);
    if constexpr (ROWMIN) return launch_rows2_64_rowmin(ix, d, rowmin, s);
    else return launch_rows2_64(ix, d, thr, rc, s, int64_t(1) << 40);
  }
  // every other form below needs a point-major copy or D <= 32
  if (!ix.xT && ix.D > 32) return launch_wide64(ix, d, thr, rc, rowmin, ROWMIN, s);
  const int64_t gy = (ndiag + kDiagBlock - 1) / kDiagBlock;
  for (int64_t y0 = 0; y0 < gy; y0 += 65535) {
  dim3 grid{unsigned((ix.M + kSeg - 1) / kSeg), unsigned(std::min<int64_t>(65535, gy - y0)), 1u};
  if (ix.xT && ix.Dp == 4 && ix.has_lo)
    MOMENTI_LAUNCH("allpairs", s, k_allpairs_pm<4, true, ROWMIN><<<grid, kDiagBlock, 0, s>>>(ix, d, thr, rc, rowmin, y0));
  else if (ix.xT && ix.Dp == 4 && rows_fit(ix.w, 4)) {
    const size_t smem = rows_smem(ix.w, 4);
    cudaError_t e = allow_smem(reinterpret_cast<const void*>(k_allpairs_rows<4, ROWMIN>), smem);
    if (e != cudaSuccess) return e;
    MOMENTI_LAUNCH("allpairs", s, k_allpairs_rows<4, ROWMIN><<<grid, kDiagBlock, smem, s>>>(ix, d, thr, rc, rowmin, y0));
  }
  else if (ix.xT && ix.Dp == 8 && ix.has_lo)
    MOMENTI_LAUNCH("allpairs", s, k_allpairs_pm<8, true, ROWMIN><<<grid, kDiagBlock, 0, s>>>(ix, d, thr, rc, rowmin, y0));
  else if (ix.xT && ix.Dp == 8 && rows_fit(ix.w, 8)) {
    const size_t smem = rows_smem(ix.w, 8);
    cudaError_t e = allow_smem(reinterpret_cast<const void*>(k_allpairs_rows<8, ROWMIN>), smem);
    if (e != cudaSuccess) return e;
    MOMENTI_LAUNCH("allpairs", s, k_allpairs_rows<8, ROWMIN><<<grid, kDiagBlock, smem, s>>>(ix, d, thr, rc, rowmin, y0));
  }
  else if (ix.xT && ix.Dp == 16 && ix.has_lo)
    MOMENTI_LAUNCH("allpairs", s, k_allpairs_pm<16, true, ROWMIN><<<grid, kDiagBlock, 0, s>>>(ix, d, thr, rc, rowmin, y0));
  else if (ix.xT && ix.Dp == 16 && rows_fit(ix.w, 16)) {
    const size_t smem = rows_smem(ix.w, 16);
    cudaError_t e = allow_smem(reinterpret_cast<const void*>(k_allpairs_rows<16, ROWMIN>), smem);
    if (e != cudaSuccess) return e;
    MOMENTI_LAUNCH("allpairs", s, k_allpairs_rows<16, ROWMIN><<<grid, kDiagBlock, smem, s>>>(ix, d, thr, rc, rowmin, y0));
  }
  else if (ix.D <= 16)
    MOMENTI_LAUNCH("allpairs", s, k_allpairs<16, ROWMIN><<<grid, kDiagBlock, 0, s>>>(ix, d, thr, rc, rowmin, y0));
  else {
    const size_t smem = size_t(32) * (kDiagBlock + 1) * sizeof(float);
    cudaError_t e = allow_smem(reinterpret_cast<const void*>(k_allpairs_wide<32, ROWMIN>), smem);
    if (e != cudaSuccess) return e;
    MOMENTI_LAUNCH("allpairs", s, k_allpairs_wide<32, ROWMIN><<<grid, kDiagBlock, smem, s>>>(ix, d, thr, rc, rowmin, y0));
  }
  }
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_verify_events(const Index& ix, int d, const HashSet& hs,
                                 const CollideScratch& cs, float tau, PairRec* rec,
                                 uint64_t rec_cap, cudaStream_t s) {
#define MOMENTI_VE(DM, PM, LO) MOMENTI_LAUNCH("verify_events", s, k_verify_events<DM, PM, LO><<<sm_count() * 8, 256, 0, s>>>(ix, d, hs, cs.events, cs.counters, cs.ev_cap, tau, rec, rec_cap))
  const bool lo = ix.has_lo;
  if (ix.xT && ix.Dp == 4) { if (lo) MOMENTI_VE(4, true, true); else MOMENTI_VE(4, true, false); }
  else if (ix.xT && ix.Dp == 8) { if (lo) MOMENTI_VE(8, true, true); else MOMENTI_VE(8, true, false); }
  else if (ix.xT && ix.Dp == 16) { if (lo) MOMENTI_VE(16, true, true); else MOMENTI_VE(16, true, false); }
  else if (ix.D <= 16) MOMENTI_VE(16, false, false);
  else MOMENTI_VE(0, false, false);
#undef MOMENTI_VE
  return cudaGetLastError();
}

cudaError_t launch_verify_pairs(const Index& ix, int d, const uint64_t* pairs, int64_t m,
                                int fp64, double* per_dim, double* dist_d, uint64_t* dims,
                                cudaStream_t s) {
  if (m <= 0) return cudaSuccess;
  int64_t g = (m + 7) / 8;
  if (g > sm_count() * 16) g = sm_count() * 16;
  MOMENTI_LAUNCH("verify_pairs", s, k_verify_pairs<<<unsigned(g), 256, 0, s>>>(ix, d, pairs, m, fp64, per_dim, dist_d, dims));
  return cudaGetLastError();
}

// Recorded pairs whose approximate distance lies in (lo, hi], compacted.
__global__ void k_select_pairs(const uint64_t* __restrict__ pairs, const float* __restrict__ dd,
                               uint64_t m, float lo, float hi, uint64_t* __restrict__ out,
                               unsigned long long* __restrict__ count) {
  const int lane = threadIdx.x & 31;
  for (uint64_t q0 = blockIdx.x * uint64_t(blockDim.x); q0 < m; q0 += uint64_t(gridDim.x) * blockDim.x) {
    const uint64_t q = q0 + threadIdx.x;
    const bool keep = q < m && dd[q] > lo && dd[q] <= hi;
    const unsigned mask = __ballot_sync(0xffffffffu, keep);
    if (!mask) continue;
    unsigned long long base = 0;
    if (lane == __ffs(mask) - 1) base = atomicAdd(count, (unsigned long long)__popc(mask));
    base = __shfl_sync(0xffffffffu, base, __ffs(mask) - 1);
    if (keep) out[base + __popc(mask & ((1u << lane) - 1u))] = pairs[q];
  }
}

cudaError_t launch_select_pairs(const uint64_t* pairs, const float* dd, uint64_t m, float lo,
                                float hi, uint64_t* out, unsigned long long* count, cudaStream_t s) {
  if (m == 0) return cudaSuccess;
  uint64_t g = (m + 255) / 256;
  if (g > sm_count() * 8) g = sm_count() * 8;
  MOMENTI_LAUNCH("select_pairs", s, k_select_pairs<<<unsigned(g), 256, 0, s>>>(pairs, dd, m, lo, hi, out, count));
  return cudaGetLastError();
}

cudaError_t launch_allpairs(const Index& ix, int d, float thr, const ApRec& rc, cudaStream_t s) {
  return allpairs_dispatch<false>(ix, d, thr, rc, nullptr, s);
}

cudaError_t launch_allpairs_rowmin(const Index& ix, int d, float* rowmin, cudaStream_t s) {
  return allpairs_dispatch<true>(ix, d, 0.f, ApRec{}, rowmin, s);
}

}  // namespace momenti
