// Index construction of Section 4: for every (repetition j, dimension f)
// the windows ordered lexicographically by their K-value hash strings, so
// that every prefix length i groups colliding windows into contiguous runs.
//
// A batched, stable least-significant-digit radix sort over the K key bytes
// (8-bit digits, last concatenation first), one segment per (j, f), all
// segments of a batch of repetitions in the same launches.  Each pass is
// three kernels: per-tile digit histograms, a per-segment scan of
// (digit, tile) counts, and a stable scatter that ranks equal digits with
// warp-level match masks and writes each tile in digit order through
// shared memory, so that equal digits leave as contiguous runs.  The final
// kernel writes the sorted window order
// and, per rank, the number of hash values shared with the previous rank
// (the longest common prefix, 0..K), which is all the traversal needs.
#include "internal.h"

#include <algorithm>

namespace momenti {

namespace {

constexpr int kThreads = 256;
constexpr int kItems = 8;                      // per thread
constexpr int kTile = kThreads * kItems;       // 2048 entries per CTA
constexpr int kWarps = kThreads / 32;
constexpr int kWarpSpan = kTile / kWarps;      // 256 entries per warp
constexpr int kRounds = kWarpSpan / 32;        // 8

struct Src {
  // pass 0 reads keys [j][a][f] and the implicit value a; later passes read
  // the ping-pong buffers [seg][M]
  const uint64_t* keys;
  const uint64_t* kin;
  const uint32_t* vin;
  int64_t M;
  int D, j0;
  bool first;
  __device__ __forceinline__ uint64_t load_key(int seg, int64_t p) const {
    if (first) {
      int j = j0 + seg / D, f = seg - (seg / D) * D;
      return keys[(int64_t(j) * M + p) * D + f];
    }
    return kin[int64_t(seg) * M + p];
  }
  __device__ __forceinline__ void load(int seg, int64_t p, uint64_t& k, uint32_t& v) const {
    if (first) {
      int j = j0 + seg / D, f = seg - (seg / D) * D;
      k = keys[(int64_t(j) * M + p) * D + f];
      v = uint32_t(p);
    } else {
      k = kin[int64_t(seg) * M + p];
      v = vin[int64_t(seg) * M + p];
    }
  }
};

__global__ void __launch_bounds__(kThreads)
k_hist(Src src, int shift, int tiles, uint32_t* __restrict__ hist) {
  __shared__ uint32_t h[256];
  // segments fastest: the first pass reads [j][a][0..D) rows of all dims together
  const int seg = blockIdx.x, tile = blockIdx.y;
  for (int d = threadIdx.x; d < 256; d += kThreads) h[d] = 0;
  __syncthreads();
  const int64_t base = int64_t(tile) * kTile;
  uint64_t k[kItems];
#pragma unroll
  for (int r = 0; r < kItems; ++r) {
    const int64_t p = base + r * kThreads + threadIdx.x;
    k[r] = p < src.M ? src.load_key(seg, p) : 0ull;
  }
#pragma unroll
  for (int r = 0; r < kItems; ++r) {
    const int64_t p = base + r * kThreads + threadIdx.x;
    if (p < src.M) atomicAdd(&h[uint32_t(k[r] >> shift) & 255u], 1u);
  }
  __syncthreads();
  uint32_t* out = hist + int64_t(seg) * 256 * tiles;
  for (int d = threadIdx.x; d < 256; d += kThreads) out[int64_t(d) * tiles + tile] = h[d];
}

// Exclusive scan over the digit-major (digit, tile) counts of one segment.
__global__ void __launch_bounds__(256) k_scan(int tiles, uint32_t* __restrict__ hist) {
  __shared__ uint32_t tot[256];
  const int seg = blockIdx.x, d = threadIdx.x;
  uint32_t* hs = hist + int64_t(seg) * 256 * tiles + int64_t(d) * tiles;
  uint32_t s = 0;
  int t0 = 0;
  for (; t0 + 8 <= tiles; t0 += 8) {          // eight independent loads in flight
    uint32_t c[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) c[q] = hs[t0 + q];
#pragma unroll
    for (int q = 0; q < 8; ++q) s += c[q];
  }
  for (; t0 < tiles; ++t0) s += hs[t0];
  tot[d] = s;
  __syncthreads();
  // Hillis-Steele inclusive scan of the 256 digit totals
  for (int off = 1; off < 256; off <<= 1) {
    uint32_t v = d >= off ? tot[d - off] : 0u;
    __syncthreads();
    tot[d] += v;
    __syncthreads();
  }
  uint32_t run = tot[d] - s;   // exclusive
  int t1 = 0;
  for (; t1 + 8 <= tiles; t1 += 8) {
    uint32_t c[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) c[q] = hs[t1 + q];
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      hs[t1 + q] = run;
      run += c[q];
    }
  }
  for (; t1 < tiles; ++t1) {
    uint32_t c = hs[t1];
    hs[t1] = run;
    run += c;
  }
}

__global__ void __launch_bounds__(kThreads)
k_scatter(Src src, int shift, int tiles, const uint32_t* __restrict__ hist,
          uint64_t* __restrict__ kout, uint32_t* __restrict__ vout) {
  __shared__ uint32_t wh[kWarps][256];
  __shared__ uint32_t loff[256];             // tile-local start of each digit
  __shared__ uint64_t sk[kTile];             // the tile in digit order
  __shared__ uint32_t sv[kTile];
  const int seg = blockIdx.x, tile = blockIdx.y;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int q = threadIdx.x; q < kWarps * 256; q += kThreads) (&wh[0][0])[q] = 0;
  __syncthreads();
  const int64_t base = int64_t(tile) * kTile + int64_t(warp) * kWarpSpan;
  const uint32_t lt = (1u << lane) - 1u;
  uint64_t key[kRounds];
  uint32_t val[kRounds], dig[kRounds], loc[kRounds];
  // all loads of the warp's span first (independent, in flight together)
#pragma unroll
  for (int r = 0; r < kRounds; ++r) {
    const int64_t p = base + r * 32 + lane;
    key[r] = 0;
    val[r] = 0;
    if (p < src.M) src.load(seg, p, key[r], val[r]);
  }
#pragma unroll
  for (int r = 0; r < kRounds; ++r) {
    const int64_t p = base + r * 32 + lane;
    // out of range: a digit no valid item has
    const uint32_t dg = p < src.M ? uint32_t(key[r] >> shift) & 255u : 256u + lane;
    dig[r] = dg;
    uint32_t peers = __match_any_sync(0xffffffffu, dg);
    uint32_t rank = __popc(peers & lt);
    uint32_t cnt = __popc(peers);
    uint32_t b = 0;
    if (dg < 256u) b = wh[warp][dg];
    __syncwarp();
    if (dg < 256u && rank == 0) wh[warp][dg] = b + cnt;
    __syncwarp();
    loc[r] = b + rank;
  }
  __syncthreads();
  for (int d = threadIdx.x; d < 256; d += kThreads) {
    uint32_t run = 0;
    for (int w = 0; w < kWarps; ++w) {
      uint32_t c = wh[w][d];
      wh[w][d] = run;
      run += c;
    }
    loff[d] = run;                           // digit total, scanned below
  }
  __syncthreads();
  if (threadIdx.x < 32) {                    // exclusive scan of the 256 totals
    uint32_t v[8], run = 0;
#pragma unroll
    for (int q = 0; q < 8; ++q) { v[q] = loff[lane * 8 + q]; run += v[q]; }
    uint32_t incl = run;
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t u = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += u;
    }
    uint32_t b = incl - run;
#pragma unroll
    for (int q = 0; q < 8; ++q) { loff[lane * 8 + q] = b; b += v[q]; }
  }
  __syncthreads();
  // the tile in digit order in shared memory (stable within each digit) ...
#pragma unroll
  for (int r = 0; r < kRounds; ++r) {
    if (dig[r] < 256u) {
      const uint32_t q = loff[dig[r]] + wh[warp][dig[r]] + loc[r];
      sk[q] = key[r];
      sv[q] = val[r];
    }
  }
  __syncthreads();
  // ... then written out in that order: runs of equal digits are contiguous
  const uint32_t* hs = hist + int64_t(seg) * 256 * tiles;
  const int64_t n_tile = min(int64_t(kTile), src.M - int64_t(tile) * kTile);
  for (int q = threadIdx.x; q < n_tile; q += kThreads) {
    const uint64_t k = sk[q];
    const uint32_t d = uint32_t(k >> shift) & 255u;
    const uint32_t dst = hs[int64_t(d) * tiles + tile] + (uint32_t(q) - loff[d]);
    kout[int64_t(seg) * src.M + dst] = k;
    vout[int64_t(seg) * src.M + dst] = sv[q];
  }
}

__global__ void k_finish(const uint64_t* __restrict__ kin, const uint32_t* __restrict__ vin,
                         int64_t M, int D, int j0, int segs, int K, uint32_t* __restrict__ order,
                         uint8_t* __restrict__ lcp) {
  int64_t total = int64_t(segs) * M;
  for (int64_t q = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; q < total;
       q += int64_t(gridDim.x) * blockDim.x) {
    int64_t seg = q / M, p = q - seg * M;
    int64_t j = j0 + seg / D, f = seg % D;
    int64_t o = (j * D + f) * M + p;
    order[o] = vin[q];
    uint32_t l = 0;
    if (p > 0) {
      uint64_t x = kin[q] ^ kin[q - 1];
      l = x == 0 ? 8u : uint32_t(__clzll(x)) / 8u;
      if (l > uint32_t(K)) l = uint32_t(K);
    }
    lcp[o] = uint8_t(l);
  }
}

}  // namespace

int64_t sort_hist_entries(int64_t M, int segs) {
  int64_t tiles = (M + kTile - 1) / kTile;
  return int64_t(segs) * 256 * tiles;
}

cudaError_t launch_sort_reps(const Index& ix, int j0, int j1, const SortScratch& sc,
                             cudaStream_t s) {
  if (j1 <= j0) return cudaSuccess;
  const int segs = (j1 - j0) * ix.D;
  if (int64_t(segs) * ix.M > sc.cap_entries || sort_hist_entries(ix.M, segs) > sc.hist_entries)
    return cudaErrorInvalidValue;
  const int tiles = int((ix.M + kTile - 1) / kTile);
  dim3 grid{unsigned(segs), unsigned(tiles), 1u};
  uint64_t* kb[2] = {sc.k0, sc.k1};
  uint32_t* vb[2] = {sc.v0, sc.v1};
  for (int pass = 0; pass < ix.K; ++pass) {
    const int byte = ix.K - 1 - pass;          // 0 = most significant hash value
    const int shift = 56 - 8 * byte;
    Src src{ix.keys, pass ? kb[(pass - 1) & 1] : nullptr, pass ? vb[(pass - 1) & 1] : nullptr,
            ix.M, ix.D, j0, pass == 0};
    MOMENTI_LAUNCH("sort_hist", s, k_hist<<<grid, kThreads, 0, s>>>(src, shift, tiles, sc.hist));
    MOMENTI_LAUNCH("sort_scan", s, k_scan<<<segs, 256, 0, s>>>(tiles, sc.hist));
    MOMENTI_LAUNCH("sort_scatter", s, k_scatter<<<grid, kThreads, 0, s>>>(src, shift, tiles, sc.hist, kb[pass & 1], vb[pass & 1]));
  }
  const int last = (ix.K - 1) & 1;
  int64_t total = int64_t(segs) * ix.M;
  int g = int(std::min<int64_t>((total + 255) / 256, 152 * 64));
  MOMENTI_LAUNCH("sort_finish", s, k_finish<<<g, 256, 0, s>>>(kb[last], vb[last], ix.M, ix.D, j0, segs, ix.K, ix.order, ix.lcp));
  return cudaGetLastError();
}

}  // namespace momenti
