// Index construction of Section 4: for every (repetition j, dimension f)
// the windows ordered lexicographically by their K-value hash strings, so
// that every prefix length i groups colliding windows into contiguous runs.
//
// A most-significant-digit radix partition followed by shared-memory
// sorts.  Level t (t = 0, 1, ...) partitions ranges ("items") stably by
// hash value t (one byte of the big-endian composite key); a partition
// never moves an entry out of its item, so every entry lands in its final
// position's bucket.  Buckets of at most kLocalMax entries are packed, in
// order, into chunks that one CTA then sorts completely in shared memory
// (a stable least-significant-digit sort over the bytes that vary inside
// the chunk); larger buckets become the items of level t + 1.  After level
// K - 1 every bucket holds equal keys and is already in order.  On the
// hash strings of z-normalised windows one level usually suffices: the
// largest bucket of the first hash value holds a few percent of the
// windows.
//
// Each level is three kernels: per-tile digit histograms, a per-item scan
// of (digit, tile) counts that also classifies the buckets (chunks for the
// shared-memory sort, items for the next level), and a stable scatter that
// ranks equal digits with warp match masks and writes each tile in digit
// order through shared memory.  The final kernel writes, per rank, the
// sorted window and the number of hash values shared with the previous
// rank (the longest common prefix, 0..K), which is all the traversal needs.
//
// Every kernel reads its work counts from device counters (grid-stride
// loops), so the levels can run without the host: the index build reads
// the counts after each level to size the next launch exactly, the
// allocation-free entry point launches all K levels with fixed grids.
#include "internal.h"

#include <algorithm>

namespace momenti {

namespace {

constexpr int kThreads = 256;
constexpr int kItems = 8;                      // per thread
constexpr int kTile = kSortTile;               // entries per partition tile
static_assert(kTile == kThreads * kItems, "partition tile");
constexpr int kWarps = kThreads / 32;
constexpr int kWarpSpan = kTile / kWarps;      // 256 entries per warp
constexpr int kRounds = kWarpSpan / 32;        // 8

constexpr int kLocalThreads = 128;
constexpr int kLocalWarps = kLocalThreads / 32;
constexpr int kLocalRounds = kSortLocalMax / (kLocalWarps * 32);   // 16
static_assert(kSortLocalMax <= 65536, "chunk ranks travel as 16-bit values");

// counters: [2 t] items and [2 t + 1] tiles of level t (t = 0..8), then
constexpr int kCntChunks = 20;   // chunks for the shared-memory sort
constexpr int kCntOverflow = 22; // a capacity was exceeded

struct Level {
  // level 0 reads keys [j][a][f] and the implicit value a; later levels
  // read the ping-pong buffers [seg][M]
  const uint64_t* keys;
  const uint64_t* kin;
  const uint32_t* vin;
  uint64_t* kout;
  uint32_t* vout;
  int64_t M;
  int D, j0, t, K, segs;
  const SortItem* items;
  SortItem* items_next;
  const uint64_t* tile_item;
  uint64_t* tile_next;
  uint32_t* hist;
  SortChunk* chunks;
  uint32_t* cnt;
  uint32_t item_cap, tile_cap, chunk_cap;
  __device__ __forceinline__ uint64_t load_key(uint32_t seg, int64_t p) const {
    if (t == 0) {
      const int j = j0 + int(seg) / D, f = int(seg) - (int(seg) / D) * D;
      return keys[(int64_t(j) * M + p) * D + f];
    }
    return kin[int64_t(seg) * M + p];
  }
  __device__ __forceinline__ void load(uint32_t seg, int64_t p, uint64_t& k, uint32_t& v) const {
    if (t == 0) {
      k = load_key(seg, p);
      v = uint32_t(p);
    } else {
      k = kin[int64_t(seg) * M + p];
      v = vin[int64_t(seg) * M + p];
    }
  }
  __device__ __forceinline__ uint32_t digit(uint64_t k) const {
    return uint32_t(k >> (56 - 8 * t)) & 255u;
  }
  // the item of a launch tile, false for an entry that is not a valid tile of
  // a valid item (only after an overflow; nothing outside the buffers is read)
  __device__ __forceinline__ bool tile_of(uint32_t tile, SortItem& it, uint32_t& tt) const {
    const uint64_t te = tile_item[tile];
    const uint32_t ii = uint32_t(te);
    tt = uint32_t(te >> 32);
    if (ii >= min(cnt[2 * t], item_cap)) return false;
    it = items[ii];
    return it.seg < uint32_t(segs) && int64_t(it.start) + it.size <= M &&
           tt < (it.size + kTile - 1) / kTile &&
           int64_t(it.hist0) + (it.size + kTile - 1) / kTile <= int64_t(tile_cap);
  }
};

__device__ __forceinline__ uint32_t ntiles(uint32_t size) { return (size + kTile - 1) / kTile; }

// Level 0: one item per segment.
// Launch tiles run segment-fastest, so that the D segments of a repetition,
// which read the same rows of the key array, are processed together.
__global__ void k_sort_init(int segs, int64_t M, SortItem* items, uint64_t* tile_item,
                            uint32_t* cnt) {
  const uint32_t tpm = uint32_t((M + kTile - 1) / kTile);
  const int64_t total = int64_t(segs) * tpm;
  for (int64_t q = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; q < total;
       q += int64_t(gridDim.x) * blockDim.x) {
    const uint32_t seg = uint32_t(q % segs), tt = uint32_t(q / segs);
    tile_item[q] = (uint64_t(tt) << 32) | seg;
    if (tt == 0) items[seg] = SortItem{seg, 0u, uint32_t(M), seg * tpm, 0u, {0u, 0u, 0u}};
  }
  if (blockIdx.x == 0 && threadIdx.x < 32) {
    for (int c = threadIdx.x; c < 32; c += 32) cnt[c] = 0;
    __syncwarp();
    if (threadIdx.x == 0) {
      cnt[0] = uint32_t(segs);
      cnt[1] = uint32_t(total);
    }
  }
}

__global__ void __launch_bounds__(kThreads) k_sort_hist(Level lv) {
  __shared__ uint32_t h[256];
  // the next level's counts start from zero (its items are added by the
  // scan kernel of this level, which runs after this one)
  if (blockIdx.x == 0 && threadIdx.x < 2 && lv.t < 8) lv.cnt[2 * (lv.t + 1) + threadIdx.x] = 0;
  const uint32_t nt = min(lv.cnt[2 * lv.t + 1], lv.tile_cap);
  for (uint32_t tile = blockIdx.x; tile < nt; tile += gridDim.x) {
    SortItem it;
    uint32_t tt;
    if (!lv.tile_of(tile, it, tt)) continue;
    for (int d = threadIdx.x; d < 256; d += kThreads) h[d] = 0;
    __syncthreads();
    const int64_t base = int64_t(it.start) + int64_t(tt) * kTile;
    const int64_t end = int64_t(it.start) + it.size;
    uint64_t k[kItems];
#pragma unroll
    for (int r = 0; r < kItems; ++r) {
      const int64_t p = base + r * kThreads + threadIdx.x;
      k[r] = p < end ? lv.load_key(it.seg, p) : 0ull;
    }
#pragma unroll
    for (int r = 0; r < kItems; ++r) {
      const int64_t p = base + r * kThreads + threadIdx.x;
      if (p < end) atomicAdd(&h[lv.digit(k[r])], 1u);
    }
    __syncthreads();
    const uint32_t nti = ntiles(it.size);
    uint32_t* out = lv.hist + int64_t(it.hist0) * 256;
    for (int d = threadIdx.x; d < 256; d += kThreads) out[int64_t(d) * nti + tt] = h[d];
    __syncthreads();
  }
}

// Exclusive scan over the digit-major (digit, tile) counts of one item, then
// the item's buckets become chunks (at most kSortLocalMax entries, packed in
// order) or items of the next level.
__global__ void __launch_bounds__(256) k_sort_scan(Level lv) {
  __shared__ uint32_t tot[256], bstart[256];
  const uint32_t ni = min(lv.cnt[2 * lv.t], lv.item_cap);
  const int d = threadIdx.x;
  for (uint32_t item = blockIdx.x; item < ni; item += gridDim.x) {
    const SortItem it = lv.items[item];
    const uint32_t tiles = ntiles(it.size);
    if (it.seg >= uint32_t(lv.segs) || int64_t(it.start) + it.size > lv.M ||
        int64_t(it.hist0) + tiles > int64_t(lv.tile_cap))
      continue;                                   // only after an overflow
    uint32_t* hs = lv.hist + int64_t(it.hist0) * 256 + int64_t(d) * tiles;
    uint32_t s = 0;
    uint32_t t0 = 0;
    for (; t0 + 8 <= tiles; t0 += 8) {          // eight independent loads in flight
      uint32_t c[8];
#pragma unroll
      for (int q = 0; q < 8; ++q) c[q] = hs[t0 + q];
#pragma unroll
      for (int q = 0; q < 8; ++q) s += c[q];
    }
    for (; t0 < tiles; ++t0) s += hs[t0];
    tot[d] = s;
    bstart[d] = s;
    __syncthreads();
    // Hillis-Steele inclusive scan of the 256 digit totals
    for (int off = 1; off < 256; off <<= 1) {
      uint32_t v = d >= off ? bstart[d - off] : 0u;
      __syncthreads();
      bstart[d] += v;
      __syncthreads();
    }
    uint32_t run = bstart[d] - s;   // exclusive, relative to the item's start
    __syncthreads();
    bstart[d] = run;
    uint32_t t1 = 0;
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
    __syncthreads();
    if (d == 0) {
      // classification, in digit order: a bucket's first entry shares t
      // hash values with its predecessor (the item's own first entry keeps
      // the item's count).  Two walks over the digits: the first counts the
      // chunks and items this item makes, so that one atomic reserves their
      // slots; the second writes them.
      const bool last_level = lv.t + 1 >= lv.K;
      uint32_t n_chunks = 0, n_items = 0, n_tiles = 0, chunk0 = 0, item0 = 0, tile0 = 0;
      for (int pass = 0; pass < 2; ++pass) {
        uint32_t nch = 0, nit = 0, ntl = 0;
        uint32_t c_start = 0, c_size = 0, c_lcp = 0;
        bool open = false, first = true;
        auto emit = [&](uint32_t st, uint32_t sz, uint32_t l0, uint32_t equal) {
          if (pass == 1) {
            const uint32_t slot = chunk0 + nch;
            if (slot < lv.chunk_cap) {
              SortChunk ch;
              ch.seg = it.seg;
              ch.start = st;
              ch.size = sz;
              ch.lcp0 = uint8_t(l0);
              ch.buf = uint8_t(lv.t & 1);
              ch.equal = uint8_t(equal);
              ch.pad = 0;
              lv.chunks[slot] = ch;
            } else {
              lv.cnt[kCntOverflow] = 1u;
            }
          }
          ++nch;
        };
        for (int g = 0; g < 256; ++g) {
          const uint32_t sz = tot[g];
          if (!sz) continue;
          const uint32_t l0 = first ? it.lcp0 : uint32_t(lv.t);
          first = false;
          const uint32_t st = it.start + bstart[g];
          if (sz > uint32_t(kSortLocalMax)) {
            if (open) emit(c_start, c_size, c_lcp, 0u);
            open = false;
            if (last_level) {
              emit(st, sz, l0, 1u);            // equal keys: already in order
            } else {
              const uint32_t nt = ntiles(sz);
              if (pass == 1) {
                const uint32_t slot = item0 + nit, tb = tile0 + ntl;
                if (slot < lv.item_cap && tb + nt <= lv.tile_cap) {
                  lv.items_next[slot] = SortItem{it.seg, st, sz, tb, l0, {0u, 0u, 0u}};
                  for (uint32_t q = 0; q < nt; ++q) lv.tile_next[tb + q] = (uint64_t(q) << 32) | slot;
                } else {
                  lv.cnt[kCntOverflow] = 1u;
                }
              }
              ++nit;
              ntl += nt;
            }
          } else if (open && c_size + sz <= uint32_t(kSortLocalMax)) {
            c_size += sz;
          } else {
            if (open) emit(c_start, c_size, c_lcp, 0u);
            open = true;
            c_start = st;
            c_size = sz;
            c_lcp = l0;
          }
        }
        if (open) emit(c_start, c_size, c_lcp, 0u);
        if (pass == 0) {
          n_chunks = nch;
          n_items = nit;
          n_tiles = ntl;
          if (n_chunks) chunk0 = atomicAdd(&lv.cnt[kCntChunks], n_chunks);
          if (n_items) {
            item0 = atomicAdd(&lv.cnt[2 * (lv.t + 1)], n_items);
            tile0 = atomicAdd(&lv.cnt[2 * (lv.t + 1) + 1], n_tiles);
          }
        }
      }
    }
    __syncthreads();
  }
}

__global__ void __launch_bounds__(kThreads) k_sort_scatter(Level lv) {
  __shared__ uint32_t wh[kWarps][256];
  __shared__ uint32_t loff[256];             // tile-local start of each digit
  __shared__ uint64_t sk[kTile];             // the tile in digit order
  __shared__ uint32_t sv[kTile];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const uint32_t lt = (1u << lane) - 1u;
  const uint32_t nt = min(lv.cnt[2 * lv.t + 1], lv.tile_cap);
  for (uint32_t tile = blockIdx.x; tile < nt; tile += gridDim.x) {
    SortItem it;
    uint32_t tt;
    if (!lv.tile_of(tile, it, tt)) continue;
    for (int q = threadIdx.x; q < kWarps * 256; q += kThreads) (&wh[0][0])[q] = 0;
    __syncthreads();
    const int64_t end = int64_t(it.start) + it.size;
    const int64_t base = int64_t(it.start) + int64_t(tt) * kTile + int64_t(warp) * kWarpSpan;
    uint64_t key[kRounds];
    uint32_t val[kRounds], dig[kRounds], loc[kRounds];
    // all loads of the warp's span first (independent, in flight together)
#pragma unroll
    for (int r = 0; r < kRounds; ++r) {
      const int64_t p = base + r * 32 + lane;
      key[r] = 0;
      val[r] = 0;
      if (p < end) lv.load(it.seg, p, key[r], val[r]);
    }
#pragma unroll
    for (int r = 0; r < kRounds; ++r) {
      const int64_t p = base + r * 32 + lane;
      // out of range: a digit no valid entry has
      const uint32_t dg = p < end ? lv.digit(key[r]) : 256u + lane;
      dig[r] = dg;
      const uint32_t peers = __match_any_sync(0xffffffffu, dg);
      const uint32_t rank = __popc(peers & lt);
      const uint32_t cnt = __popc(peers);
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
        const uint32_t c = wh[w][d];
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
    const uint32_t nti = ntiles(it.size);
    const uint32_t* hs = lv.hist + int64_t(it.hist0) * 256;
    const int64_t n_tile = min(int64_t(kTile), end - (int64_t(it.start) + int64_t(tt) * kTile));
    const int64_t obase = int64_t(it.seg) * lv.M + it.start;
    for (int q = threadIdx.x; q < n_tile; q += kThreads) {
      const uint64_t k = sk[q];
      const uint32_t d = lv.digit(k);
      const uint32_t dst = hs[int64_t(d) * nti + tt] + (uint32_t(q) - loff[d]);
      lv.kout[obase + dst] = k;
      lv.vout[obase + dst] = sv[q];
    }
    __syncthreads();
  }
}

struct LocalArgs {
  const uint64_t* k[2];
  const uint32_t* v[2];
  const SortChunk* chunks;
  uint32_t* cnt;
  uint32_t chunk_cap;
  int64_t M;
  int D, j0, K, segs;
  uint64_t kmask;                 // the K leading bytes of a key
  uint32_t* order;
  uint8_t* lcp;
};

// Stable LSD pass of one 8-bit digit over n entries in shared memory (src ->
// dst): keys and their 16-bit ranks in the chunk move together.  Each warp
// owns a contiguous span and ranks it with match masks against its own
// digit counters; the warp-order scan of the counters keeps the pass
// stable.  Keys stay in registers between counting and scatter.
__device__ __forceinline__ void local_pass(const uint64_t* sk, const uint16_t* si, uint64_t* dk,
                                           uint16_t* di, int n, int shift, uint16_t (*wh)[256],
                                           uint32_t* doff) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const uint32_t lt = (1u << lane) - 1u;
  {
    uint32_t* z = reinterpret_cast<uint32_t*>(&wh[0][0]);
    for (int q = threadIdx.x; q < kLocalWarps * 128; q += kLocalThreads) z[q] = 0u;
  }
  // span: a multiple of 32 covering n over the warps
  const int span = ((n + kLocalWarps * 32 - 1) / (kLocalWarps * 32)) * 32;
  uint64_t key[kLocalRounds];
  uint16_t idx[kLocalRounds];
  uint32_t pk[kLocalRounds];            // digit | local rank << 9
#pragma unroll
  for (int r = 0; r < kLocalRounds; ++r) {
    const int q = warp * span + r * 32 + lane;
    const bool in = r * 32 < span && q < n;
    key[r] = in ? sk[q] : 0ull;
    idx[r] = in ? si[q] : uint16_t(0);
    pk[r] = in ? uint32_t(key[r] >> shift) & 255u : 256u + lane;
  }
  __syncthreads();
#pragma unroll
  for (int r = 0; r < kLocalRounds; ++r) {
    if (r * 32 >= span) break;                 // uniform over the block
    const uint32_t dg = pk[r];
    const uint32_t peers = __match_any_sync(0xffffffffu, dg);
    const uint32_t rank = __popc(peers & lt);
    const uint32_t b = dg < 256u ? wh[warp][dg] : 0u;
    __syncwarp();
    if (dg < 256u && rank == 0) wh[warp][dg] = uint16_t(b + __popc(peers));
    __syncwarp();
    pk[r] = dg | ((b + rank) << 9);
  }
  __syncthreads();
  for (int d = threadIdx.x; d < 256; d += kLocalThreads) {
    uint32_t run = 0;
#pragma unroll
    for (int h = 0; h < kLocalWarps; ++h) {
      const uint32_t c = wh[h][d];
      wh[h][d] = uint16_t(run);
      run += c;
    }
    doff[d] = run;
  }
  __syncthreads();
  if (threadIdx.x < 32) {
    uint32_t v[8], run = 0;
#pragma unroll
    for (int q = 0; q < 8; ++q) { v[q] = doff[lane * 8 + q]; run += v[q]; }
    uint32_t incl = run;
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t u = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += u;
    }
    uint32_t b = incl - run;
#pragma unroll
    for (int q = 0; q < 8; ++q) { doff[lane * 8 + q] = b; b += v[q]; }
  }
  __syncthreads();
#pragma unroll
  for (int r = 0; r < kLocalRounds; ++r) {
    const uint32_t dg = pk[r] & 511u;
    if (dg < 256u) {
      const uint32_t dst = doff[dg] + wh[warp][dg] + (pk[r] >> 9);
      dk[dst] = key[r];
      di[dst] = idx[r];
    }
  }
  __syncthreads();
}

// Each chunk sorted completely in shared memory, then order and common-
// prefix lengths written to their final ranks.  The keys of a chunk are
// first compressed without changing their order: every hash value is
// replaced by its offset from the chunk's smallest value at that position,
// in as many bits as the chunk's range there needs, and the fields are
// concatenated, first hash value most significant; the digit passes then
// run over the bits the chunk actually uses.  Two keys share a hash value
// iff they share its field, so the common-prefix length is read off the
// compressed keys: the field of their highest differing bit.
__global__ void __launch_bounds__(kLocalThreads, 5) k_sort_local(LocalArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  uint64_t* sk0 = reinterpret_cast<uint64_t*>(smem);
  uint64_t* sk1 = sk0 + kSortLocalMax;
  uint16_t* si0 = reinterpret_cast<uint16_t*>(sk1 + kSortLocalMax);
  uint16_t* si1 = si0 + kSortLocalMax;
  uint16_t (*wh)[256] = reinterpret_cast<uint16_t (*)[256]>(si1 + kSortLocalMax);
  uint32_t* doff = reinterpret_cast<uint32_t*>(&wh[kLocalWarps][0]);
  __shared__ uint32_t s_min[kLocalWarps][2], s_max[kLocalWarps][2];
  __shared__ uint32_t s_bmin[8], s_width[8], s_off[8];
  __shared__ uint8_t s_field[64];          // bit position -> hash value it belongs to
  __shared__ int s_bits;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const uint32_t nc = min(a.cnt[kCntChunks], a.chunk_cap);
  for (uint32_t c = blockIdx.x; c < nc; c += gridDim.x) {
    const SortChunk ch = a.chunks[c];
    if (ch.seg >= uint32_t(a.segs) || int64_t(ch.start) + ch.size > a.M) continue;   // only after an overflow
    const int64_t ib = int64_t(ch.seg) * a.M + ch.start;
    const int64_t ob = (int64_t(a.j0) * a.D + ch.seg) * a.M + ch.start;
    const uint64_t* kin = (ch.buf ? a.k[1] : a.k[0]) + ib;
    const uint32_t* vin = (ch.buf ? a.v[1] : a.v[0]) + ib;
    const int n = int(ch.size);
    if (ch.equal || n > kSortLocalMax) {
      // equal keys (after the last level): already in order
      for (int q = threadIdx.x; q < n; q += kLocalThreads) {
        a.order[ob + q] = vin[q];
        a.lcp[ob + q] = q == 0 ? ch.lcp0 : uint8_t(a.K);
      }
      continue;
    }
    // per-byte minimum and maximum over the chunk (four bytes per word)
    uint32_t mn[2] = {~0u, ~0u}, mx[2] = {0u, 0u};
    for (int q = threadIdx.x; q < n; q += kLocalThreads) {
      const uint64_t k = kin[q] & a.kmask;
      sk1[q] = k;                                  // the keys as loaded, for the compression
      const uint32_t w0 = uint32_t(k >> 32), w1 = uint32_t(k);
      mn[0] = __vminu4(mn[0], w0); mn[1] = __vminu4(mn[1], w1);
      mx[0] = __vmaxu4(mx[0], w0); mx[1] = __vmaxu4(mx[1], w1);
    }
    for (int off = 16; off; off >>= 1) {
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        mn[h] = __vminu4(mn[h], __shfl_xor_sync(0xffffffffu, mn[h], off));
        mx[h] = __vmaxu4(mx[h], __shfl_xor_sync(0xffffffffu, mx[h], off));
      }
    }
    if (lane == 0) {
      s_min[warp][0] = mn[0]; s_min[warp][1] = mn[1];
      s_max[warp][0] = mx[0]; s_max[warp][1] = mx[1];
    }
    __syncthreads();
    if (threadIdx.x < 8) {
      const int b = threadIdx.x, h = b >> 2, sh = 24 - 8 * (b & 3);   // byte b of the key, 0 = most significant
      uint32_t lo = 255u, hi = 0u;
      for (int w = 0; w < kLocalWarps; ++w) {
        lo = min(lo, (s_min[w][h] >> sh) & 255u);
        hi = max(hi, (s_max[w][h] >> sh) & 255u);
      }
      s_bmin[b] = lo;
      s_width[b] = hi > lo ? 32u - __clz(hi - lo) : 0u;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      int off = 0;                                  // bit offset of each field from the bottom
      for (int b = 7; b >= 0; --b) {
        s_off[b] = uint32_t(off);
        off += int(s_width[b]);
      }
      s_bits = off;
    }
    __syncthreads();
    if (threadIdx.x < 64) {
      uint8_t f = 8;
      for (int b = 0; b < 8; ++b)
        if (uint32_t(threadIdx.x) >= s_off[b] && uint32_t(threadIdx.x) < s_off[b] + s_width[b]) f = uint8_t(b);
      s_field[threadIdx.x] = f;
    }
    const uint32_t bmin_hi = (s_bmin[0] << 24) | (s_bmin[1] << 16) | (s_bmin[2] << 8) | s_bmin[3];
    const uint32_t bmin_lo = (s_bmin[4] << 24) | (s_bmin[5] << 16) | (s_bmin[6] << 8) | s_bmin[7];
    uint32_t foff[8];
#pragma unroll
    for (int b = 0; b < 8; ++b) foff[b] = s_off[b];
    for (int q = threadIdx.x; q < n; q += kLocalThreads) {
      const uint64_t k = sk1[q];
      // byte-wise offsets from the minima (no borrow: every byte is >= its minimum)
      const uint32_t d0 = __vsub4(uint32_t(k >> 32), bmin_hi), d1 = __vsub4(uint32_t(k), bmin_lo);
      uint64_t z = 0;
#pragma unroll
      for (int b = 0; b < 8; ++b) {
        const uint32_t v = ((b < 4 ? d0 : d1) >> (24 - 8 * (b & 3))) & 255u;
        z |= uint64_t(v) << foff[b];                 // width 0: the offset is 0
      }
      sk0[q] = z;
      si0[q] = uint16_t(q);
    }
    __syncthreads();
    uint64_t* ck = sk0;
    uint16_t* ci = si0;
    uint64_t* ok = sk1;
    uint16_t* oi = si1;
    const int bits = s_bits;
    for (int shift = 0; shift < bits; shift += 8) {
      local_pass(ck, ci, ok, oi, n, shift, wh, doff);
      uint64_t* tk = ck; ck = ok; ok = tk;
      uint16_t* ti = ci; ci = oi; oi = ti;
    }
    for (int q = threadIdx.x; q < n; q += kLocalThreads) {
      a.order[ob + q] = vin[ci[q]];
      uint32_t l = ch.lcp0;
      if (q > 0) {
        const uint64_t x = ck[q] ^ ck[q - 1];
        l = x == 0 ? 8u : uint32_t(s_field[63 - __clzll(x)]);
        if (l > uint32_t(a.K)) l = uint32_t(a.K);
      }
      a.lcp[ob + q] = uint8_t(l);
    }
    __syncthreads();
  }
}

constexpr size_t kLocalSmem = size_t(kSortLocalMax) * (8 + 8 + 2 + 2) +
                              size_t(kLocalWarps) * 256 * 2 + 256 * 4;

}  // namespace

SortScratch sort_scratch_carve(void* base, int64_t M, int segs) {
  const SortCaps c = sort_caps(M, segs);
  const int64_t e = M * segs;
  const auto up = sort_up256;
  unsigned char* p = static_cast<unsigned char*>(base);
  SortScratch sc;
  sc.k0 = reinterpret_cast<uint64_t*>(p); p += up(size_t(e) * 8);
  sc.k1 = reinterpret_cast<uint64_t*>(p); p += up(size_t(e) * 8);
  sc.v0 = reinterpret_cast<uint32_t*>(p); p += up(size_t(e) * 4);
  sc.v1 = reinterpret_cast<uint32_t*>(p); p += up(size_t(e) * 4);
  sc.hist = reinterpret_cast<uint32_t*>(p); p += up(size_t(c.tile_cap) * 256 * 4);
  sc.items[0] = reinterpret_cast<SortItem*>(p); p += up(size_t(c.item_cap) * sizeof(SortItem));
  sc.items[1] = reinterpret_cast<SortItem*>(p); p += up(size_t(c.item_cap) * sizeof(SortItem));
  sc.tile_item[0] = reinterpret_cast<uint64_t*>(p); p += up(size_t(c.tile_cap) * 8);
  sc.tile_item[1] = reinterpret_cast<uint64_t*>(p); p += up(size_t(c.tile_cap) * 8);
  sc.chunks = reinterpret_cast<SortChunk*>(p); p += up(size_t(c.chunk_cap) * sizeof(SortChunk));
  sc.cnt = reinterpret_cast<uint32_t*>(p);
  sc.cap_entries = e;
  sc.caps = c;
  sc.M = M;
  sc.segs = segs;
  return sc;
}

cudaError_t launch_sort_reps(const Index& ix, int j0, int j1, const SortScratch& sc,
                             cudaStream_t s) {
  if (j1 <= j0) return cudaSuccess;
  const int segs = (j1 - j0) * ix.D;
  if (sc.M != ix.M || segs > sc.segs) return cudaErrorInvalidValue;
  const SortCaps& c = sc.caps;
  cudaError_t e = allow_smem(reinterpret_cast<const void*>(k_sort_local), kLocalSmem);
  if (e != cudaSuccess) return e;
  const int64_t tpm = (ix.M + kTile - 1) / kTile;
  const int sm = sm_count();
  {
    const int64_t total = int64_t(segs) * tpm;
    const int g = int(std::min<int64_t>((total + 255) / 256, int64_t(sm) * 8));
    MOMENTI_LAUNCH("sort_init", s, k_sort_init<<<std::max(g, 1), 256, 0, s>>>(segs, ix.M, sc.items[0], sc.tile_item[0], sc.cnt));
  }
  uint32_t n_items = uint32_t(segs), n_tiles = uint32_t(int64_t(segs) * tpm);
  const bool host = sc.host_cnt != nullptr;
  for (int t = 0; t < ix.K; ++t) {
    Level lv;
    lv.keys = ix.keys;
    lv.kin = t ? (((t - 1) & 1) ? sc.k1 : sc.k0) : nullptr;
    lv.vin = t ? (((t - 1) & 1) ? sc.v1 : sc.v0) : nullptr;
    lv.kout = (t & 1) ? sc.k1 : sc.k0;
    lv.vout = (t & 1) ? sc.v1 : sc.v0;
    lv.M = ix.M;
    lv.D = ix.D;
    lv.j0 = j0;
    lv.t = t;
    lv.K = ix.K;
    lv.segs = segs;
    lv.items = sc.items[t & 1];
    lv.items_next = sc.items[(t + 1) & 1];
    lv.tile_item = sc.tile_item[t & 1];
    lv.tile_next = sc.tile_item[(t + 1) & 1];
    lv.hist = sc.hist;
    lv.chunks = sc.chunks;
    lv.cnt = sc.cnt;
    lv.item_cap = uint32_t(c.item_cap);
    lv.tile_cap = uint32_t(c.tile_cap);
    lv.chunk_cap = uint32_t(c.chunk_cap);
    // with the host in the loop the grids are exact; without it, the
    // largest a level can need (the kernels stop at the device counts)
    const unsigned gt = unsigned(std::max<int64_t>(1, host ? n_tiles : c.tile_cap));
    const unsigned gi = unsigned(std::max<int64_t>(1, host ? n_items : c.item_cap));
    MOMENTI_LAUNCH("sort_hist", s, k_sort_hist<<<gt, kThreads, 0, s>>>(lv));
    MOMENTI_LAUNCH("sort_scan", s, k_sort_scan<<<gi, 256, 0, s>>>(lv));
    MOMENTI_LAUNCH("sort_scatter", s, k_sort_scatter<<<gt, kThreads, 0, s>>>(lv));
    if (host) {
      e = cudaMemcpyAsync(sc.host_cnt, sc.cnt, 32 * sizeof(uint32_t), cudaMemcpyDeviceToHost, s);
      if (e != cudaSuccess) return e;
      e = cudaStreamSynchronize(s);
      if (e != cudaSuccess) return e;
      if (sc.host_cnt[kCntOverflow]) return cudaErrorInvalidValue;   // capacities are bounds: not expected
      n_items = sc.host_cnt[2 * (t + 1)];
      n_tiles = sc.host_cnt[2 * (t + 1) + 1];
      if (n_items == 0) break;
    }
  }
  LocalArgs la;
  la.k[0] = sc.k0;
  la.k[1] = sc.k1;
  la.v[0] = sc.v0;
  la.v[1] = sc.v1;
  la.chunks = sc.chunks;
  la.cnt = sc.cnt;
  la.chunk_cap = uint32_t(c.chunk_cap);
  la.M = ix.M;
  la.D = ix.D;
  la.j0 = j0;
  la.K = ix.K;
  la.segs = segs;
  la.kmask = ix.K >= 8 ? ~0ull : ~((~0ull) >> (8 * ix.K));
  la.order = ix.order;
  la.lcp = ix.lcp;
  // five CTAs of 4 warps per SM (shared memory bound); chunks statically
  // interleaved over them
  MOMENTI_LAUNCH("sort_local", s, k_sort_local<<<sm * 5, kLocalThreads, kLocalSmem, s>>>(la));
  return cudaGetLastError();
}

}  // namespace momenti
