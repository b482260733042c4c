// Index traversal of Algorithm 1 (the collision count W per pair) on the sorted index: at
// prefix length i, in repetition j, every pair of windows sharing the
// length-i prefix in some dimension is a collision; W(a, b) is the number
// of dimensions in which they collide, and pairs with W >= d become
// candidates.  As in Section 6.2 ("comparisons on the fly"), W is computed
// when a collision is seen, from the keys of the two windows in all D
// dimensions, so no quadratic W table is kept.  De-duplication that leaves
// the candidate set of Algorithm 1 unchanged:
//   - a pair is handled only from its lowest colliding dimension;
//   - a pair already colliding in >= d dimensions at prefix i+1 in the same
//     repetition was a candidate then (Section 6.2, duplicate collisions);
//   - a device hash set of every pair seen so far keeps each pair's first
//     (i, j) and lets only new pairs reach verification.
//
// Enumeration: within one (j, f) segment the windows of a bucket are a run
// of ranks p with lcp[p] >= i after the run's first rank.  Ranks are cut in
// chunks of 32; a tile is a pair of chunks (c1 <= c2) that can hold two
// ranks of one bucket, handled by one warp with both chunks' keys in shared
// memory.  The tiles of a launch are numbered through a scan, so work is
// balanced however skewed the bucket sizes are.
#include "internal.h"

#include <algorithm>

namespace momenti {

namespace {

constexpr uint64_t kEmpty = kSetEmpty;
constexpr int kMaxProbe = kSetMaxProbe;

struct Seg {
  int64_t M;
  int D, j0, C;
  __device__ __forceinline__ int64_t base(int seg) const {
    int j = j0 + seg / D, f = seg - (seg / D) * D;
    return (int64_t(j) * D + f) * M;
  }
};

// One warp per (segment, chunk): the last bucket start in the chunk (or -1)
// and whether any rank of the chunk continues the bucket of its predecessor.
__global__ void k_chunk_agg(const uint8_t* __restrict__ lcp, Seg sg, int segs, int i, int d,
                            int32_t* __restrict__ cagg, uint64_t* __restrict__ ntile) {
  const int64_t gw = (blockIdx.x * int64_t(blockDim.x) + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (gw >= int64_t(segs) * sg.C) return;
  const int seg = int(gw / sg.C);
  const int64_t c = gw - int64_t(seg) * sg.C;
  const uint8_t* L = lcp + sg.base(seg);
  const int64_t p = c * 32 + lane;
  const bool valid = p < sg.M;
  const int l = valid ? int(L[p]) : 0;
  const unsigned st = __ballot_sync(0xffffffffu, valid && l < i);
  // a pair handled from dim f needs d - 1 more colliding dims above f
  const int f = seg - (seg / sg.D) * sg.D;
  const bool useful = f <= sg.D - d;
  const unsigned jn = __ballot_sync(0xffffffffu, valid && l >= i && useful);
  if (lane == 0) {
    cagg[gw] = st ? int32_t(c * 32 + 31 - __clz(int(st))) : -1;
    ntile[gw] = jn ? 1u : 0u;
  }
}

// One block per segment: bucket start of each chunk's first rank (exclusive
// max-scan of the chunk aggregates) and the number of tiles whose column
// chunk is this chunk: row chunks from the bucket start's chunk up to itself.
__global__ void __launch_bounds__(1024)
k_chunk_scan(const uint8_t* __restrict__ lcp, Seg sg, int i, const int32_t* __restrict__ cagg,
             int32_t* __restrict__ cbs, uint64_t* __restrict__ ntile) {
  __shared__ int32_t wtot[32];
  __shared__ int32_t carry_s;
  const int seg = blockIdx.x;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const uint8_t* L = lcp + sg.base(seg);
  const int64_t off = int64_t(seg) * sg.C;
  if (threadIdx.x == 0) carry_s = -1;
  __syncthreads();
  for (int64_t b0 = 0; b0 < sg.C; b0 += blockDim.x) {
    const int64_t c = b0 + threadIdx.x;
    int32_t v = c < sg.C ? cagg[off + c] : -1;
    int32_t incl = v;
    for (int o = 1; o < 32; o <<= 1) {
      int32_t u = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl = max(incl, u);
    }
    if (lane == 31) wtot[wid] = incl;
    __syncthreads();
    if (wid == 0) {
      int32_t t = wtot[lane];
      for (int o = 1; o < 32; o <<= 1) {
        int32_t u = __shfl_up_sync(0xffffffffu, t, o);
        if (lane >= o) t = max(t, u);
      }
      wtot[lane] = t;
    }
    __syncthreads();
    const int32_t carry = carry_s;
    int32_t before = wid ? wtot[wid - 1] : -1;
    int32_t excl = __shfl_up_sync(0xffffffffu, incl, 1);
    if (lane == 0) excl = -1;
    excl = max(max(excl, before), carry);
    if (c < sg.C) {
      const int64_t p0 = c * 32;
      const int32_t bs = (int(L[p0]) < i) ? int32_t(p0) : excl;
      cbs[off + c] = bs;
      const uint64_t has = ntile[off + c];
      ntile[off + c] = has ? uint64_t(c - bs / 32 + 1) : 0u;
    }
    __syncthreads();
    if (threadIdx.x == 0) carry_s = max(carry, wtot[31]);
    __syncthreads();
  }
}

// Device-wide exclusive scan of n uint64 values in place; v[n] = total.
constexpr int kScanBlock = 1024;
__global__ void __launch_bounds__(kScanBlock)
k_scan_local(uint64_t* __restrict__ v, int64_t n, uint64_t* __restrict__ bsum) {
  __shared__ uint64_t wt[32];
  const int64_t q = blockIdx.x * int64_t(kScanBlock) + threadIdx.x;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  uint64_t x = q < n ? v[q] : 0;
  uint64_t incl = x;
  for (int o = 1; o < 32; o <<= 1) {
    uint64_t u = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += u;
  }
  if (lane == 31) wt[wid] = incl;
  __syncthreads();
  if (wid == 0) {
    uint64_t t = wt[lane];
    for (int o = 1; o < 32; o <<= 1) {
      uint64_t u = __shfl_up_sync(0xffffffffu, t, o);
      if (lane >= o) t += u;
    }
    wt[lane] = t;
  }
  __syncthreads();
  uint64_t before = wid ? wt[wid - 1] : 0;
  if (q < n) v[q] = before + incl - x;
  if (threadIdx.x == kScanBlock - 1) bsum[blockIdx.x] = before + incl;
}

__global__ void __launch_bounds__(kScanBlock)
k_scan_top(uint64_t* __restrict__ bsum, int64_t nb, uint64_t* __restrict__ total_out) {
  __shared__ uint64_t wt[32];
  __shared__ uint64_t carry_s;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (threadIdx.x == 0) carry_s = 0;
  __syncthreads();
  for (int64_t b0 = 0; b0 < nb; b0 += kScanBlock) {
    const int64_t q = b0 + threadIdx.x;
    uint64_t x = q < nb ? bsum[q] : 0;
    uint64_t incl = x;
    for (int o = 1; o < 32; o <<= 1) {
      uint64_t u = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += u;
    }
    if (lane == 31) wt[wid] = incl;
    __syncthreads();
    if (wid == 0) {
      uint64_t t = wt[lane];
      for (int o = 1; o < 32; o <<= 1) {
        uint64_t u = __shfl_up_sync(0xffffffffu, t, o);
        if (lane >= o) t += u;
      }
      wt[lane] = t;
    }
    __syncthreads();
    const uint64_t carry = carry_s;
    uint64_t before = wid ? wt[wid - 1] : 0;
    if (q < nb) bsum[q] = carry + before + incl - x;
    __syncthreads();
    if (threadIdx.x == 0) carry_s = carry + wt[31];
    __syncthreads();
  }
  if (threadIdx.x == 0) *total_out = carry_s;
}

__global__ void k_scan_add(uint64_t* __restrict__ v, int64_t n, const uint64_t* __restrict__ bsum) {
  const int64_t q = blockIdx.x * int64_t(kScanBlock) + threadIdx.x;
  if (q < n) v[q] += bsum[blockIdx.x];
}

struct CollideArgs {
  const uint32_t* order;
  const uint8_t* lcp;
  const uint64_t* keys;
  Seg sg;
  int segs, i, K, d, excl;
  const int32_t* cbs;
  const uint64_t* toff;    // exclusive scan, toff[E] = total tiles
  HashSet hs;
  Event* events;
  uint64_t ev_cap;
  unsigned long long* counters;
  uint64_t* out_pairs;
  uint64_t out_cap;
};

// true if key is in the set (read-only probe)
__device__ __forceinline__ bool set_contains(const HashSet& hs, uint64_t key) {
  uint64_t h = set_hash(key) & (hs.cap - 1);
  for (int probe = 0; probe < kMaxProbe; ++probe) {
    const uint64_t cur = hs.keys[h];
    if (cur == key) return true;
    if (cur == kEmpty) return false;
    h = (h + 1) & (hs.cap - 1);
  }
  return false;
}

// 0x80 in every byte of x that is zero (exact, no carries across bytes)
__device__ __forceinline__ uint64_t zero_bytes(uint64_t x) {
  const uint64_t L7 = 0x7F7F7F7F7F7F7F7Full;
  const uint64_t y = (x & L7) + L7;
  return ~(y | x | L7);
}

// Per warp: the 64 windows of a tile (32 row ranks, 32 column ranks) as
// byte planes: word (t, g) of a window holds byte t (hash value t) of the
// keys of dims 8g .. 8g+7, dim 8g+e in byte e.  Equality of the length-i
// prefixes of all dims of two windows is then i XORs and zero-byte masks.
// I = prefix length (compile time, so every per-hash-value loop is exact)
template <bool PLAIN, int I>
__global__ void __launch_bounds__(128) k_collide(CollideArgs g) {
  extern __shared__ uint64_t smem[];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const int D = g.sg.D;
  const int G = (D + 7) >> 3;
  const bool lvl_dup = !PLAIN && I < g.K;
  constexpr int NPMAX = (!PLAIN && I < 8) ? I + 1 : I;   // planes loaded
  const int NP = lvl_dup ? I + 1 : I;
  uint64_t* sp = smem + int64_t(wib) * (64 * G * NP + 32);
  uint32_t* sidx = reinterpret_cast<uint32_t*>(sp + 64 * G * NP);
  const int64_t E = int64_t(g.segs) * g.sg.C;
  const uint64_t T = g.toff[E];
  const uint64_t nw = uint64_t(gridDim.x) * (blockDim.x >> 5);
  const uint64_t w = uint64_t(blockIdx.x) * (blockDim.x >> 5) + wib;
  // a contiguous range of tiles per warp: one search, then a forward walk
  const uint64_t t_begin = T * w / nw, t_end = T * (w + 1) / nw;
  if (t_begin >= t_end) return;
  const uint32_t lt = (1u << lane) - 1u;
  auto find = [&](int64_t lo, uint64_t t) {     // largest e >= lo with toff[e] <= t
    int64_t hi = E - 1;
    while (lo < hi) {
      int64_t mid = (lo + hi + 1) >> 1;
      if (g.toff[mid] <= t) lo = mid;
      else hi = mid - 1;
    }
    return lo;
  };
  int64_t e = find(0, t_begin);
  int64_t cur = -1;
  // per column chunk state
  int j = 0, f = 0, gf = 0, ef = 0, seg = 0;
  int64_t c2 = 0;
  int32_t bs0 = 0, bs2 = 0;
  uint32_t wbl = 0;
  const uint32_t* O = nullptr;
  const uint64_t* Kj = nullptr;

  auto load_planes = [&](uint32_t win, bool ok, int r) {
    const uint64_t* kw = Kj + int64_t(win) * D;
    for (int gg = 0; gg < G; ++gg) {
      uint64_t pw[NPMAX];
#pragma unroll
      for (int q = 0; q < NPMAX; ++q) pw[q] = 0;
      for (int ee = 0; ee < 8; ++ee) {
        const int ff = gg * 8 + ee;
        if (ff >= D || !ok) break;
        const uint64_t key = kw[ff];
#pragma unroll
        for (int q = 0; q < NPMAX; ++q) pw[q] |= ((key >> (56 - 8 * q)) & 0xFFull) << (8 * ee);
      }
#pragma unroll
      for (int q = 0; q < NPMAX; ++q)
        if (q < NP) sp[(q * G + gg) * 64 + r] = pw[q];
    }
  };

  for (uint64_t t = t_begin; t < t_end; ++t) {
    if (g.toff[e + 1] <= t) {
      e = (g.toff[e + 2] <= t) ? find(e + 2, t) : e + 1;
    }
    if (e != cur) {
      // new column chunk: its ranks, keys as byte planes and bucket starts
      cur = e;
      seg = int(e / g.sg.C);
      c2 = e - int64_t(seg) * g.sg.C;
      bs0 = g.cbs[e];
      j = g.sg.j0 + seg / D;
      f = seg - (seg / D) * D;
      gf = f >> 3;
      ef = f & 7;
      const int64_t sbase = g.sg.base(seg);
      O = g.order + sbase;
      const uint8_t* Lc = g.lcp + sbase;
      Kj = g.keys + int64_t(j) * g.sg.M * D;
      const int64_t p2 = c2 * 32 + lane;
      const bool v2 = p2 < g.sg.M;
      int32_t sv = (v2 && int(Lc[p2]) < g.i) ? int32_t(p2) : -1;
      for (int o = 1; o < 32; o <<= 1) {
        int32_t u = __shfl_up_sync(0xffffffffu, sv, o);
        if (lane >= o) sv = max(sv, u);
      }
      bs2 = max(sv, bs0);
      wbl = v2 ? O[p2] : 0u;
      __syncwarp();
      sidx[32 + lane] = wbl;
      load_planes(wbl, v2, 32 + lane);
    }
    const int64_t c1 = bs0 / 32 + int64_t(t - g.toff[e]);
    const int64_t p1 = c1 * 32 + lane;
    const bool v1 = p1 < g.sg.M;
    const uint32_t wa = v1 ? O[p1] : 0u;
    __syncwarp();
    sidx[lane] = wa;
    load_planes(wa, v1, lane);
    __syncwarp();
    // row planes of this lane's window in registers (one 64-bit word per
    // hash value when D <= 8)
    uint64_t rp[I];
#pragma unroll
    for (int q = 0; q < I; ++q) rp[q] = (G == 1) ? sp[q * 64 + lane] : 0ull;
    const uint64_t valid0 = D >= 8 ? 0x8080808080808080ull
                                   : (0x8080808080808080ull & ((1ull << (8 * D)) - 1));
    const uint64_t lowmask = (gf == 0) ? ((1ull << (8 * ef)) - 1) & valid0 : 0ull;
    for (int cc = 0; cc < 32; ++cc) {
      const int64_t pc = c2 * 32 + cc;
      if (pc >= g.sg.M) break;                       // warp-uniform
      const int32_t bsc = __shfl_sync(0xffffffffu, bs2, cc);
      bool emit = p1 >= bsc && p1 < pc;
      int W = 0;
      if (emit) {
        if (G == 1) {
          uint64_t m = valid0;
#pragma unroll
          for (int q = 0; q < I; ++q) m &= zero_bytes(rp[q] ^ sp[q * 64 + 32 + cc]);
          emit = (m & lowmask) == 0;
          W = __popcll(m);
          if (emit && W >= g.d && lvl_dup) {
            const uint64_t m1 = m & zero_bytes(sp[I * 64 + lane] ^ sp[I * 64 + 32 + cc]);
            if (__popcll(m1) >= g.d) emit = false;
          }
        } else {
          bool low = false;
          for (int gg = 0; gg < G && !low; ++gg) {
            const int nvalid = min(8, D - gg * 8);
            uint64_t m = nvalid == 8 ? 0x8080808080808080ull
                                     : (0x8080808080808080ull & ((1ull << (8 * nvalid)) - 1));
#pragma unroll
            for (int q = 0; q < I; ++q)
              m &= zero_bytes(sp[(q * G + gg) * 64 + lane] ^ sp[(q * G + gg) * 64 + 32 + cc]);
            if (gg < gf) low = m != 0;
            else if (gg == gf) low = (m & ((1ull << (8 * ef)) - 1)) != 0;
            W += __popcll(m);
          }
          emit = !low;
          if (emit && W >= g.d && lvl_dup) {
            int W1 = 0;
            for (int gg = 0; gg < G; ++gg) {
              const int nvalid = min(8, D - gg * 8);
              uint64_t m = nvalid == 8 ? 0x8080808080808080ull
                                       : (0x8080808080808080ull & ((1ull << (8 * nvalid)) - 1));
#pragma unroll
              for (int q = 0; q <= I; ++q)
                m &= zero_bytes(sp[(q * G + gg) * 64 + lane] ^ sp[(q * G + gg) * 64 + 32 + cc]);
              W1 += __popcll(m);
            }
            if (W1 >= g.d) emit = false;
          }
        }
        emit = emit && W >= g.d;
      }
      uint32_t a = 0, b = 0;
      if (emit) {
        const uint32_t wb = sidx[32 + cc];
        a = min(wa, wb);
        b = max(wa, wb);
        emit = int64_t(b) - int64_t(a) > g.excl;
      }
      const uint64_t key = (uint64_t(a) << 32) | b;
      if (!PLAIN && emit) emit = !set_contains(g.hs, key);
      const unsigned m = __ballot_sync(0xffffffffu, emit);
      if (m == 0) continue;
      unsigned long long base = 0;
      if (lane == __ffs(m) - 1) base = atomicAdd(&g.counters[0], (unsigned long long)__popc(m));
      base = __shfl_sync(0xffffffffu, base, __ffs(m) - 1);
      if (emit) {
        const unsigned long long pos = base + __popc(m & lt);
        if (PLAIN) {
          if (pos < g.out_cap) g.out_pairs[pos] = key;
        } else if (pos < g.ev_cap) {
          g.events[pos] = Event{a, b, int32_t(j), 0u};
        }
      }
    }
  }
}

// ---- prefix length 1: buckets split by a second dimension ---------------

// Buckets of prefix length i (runs with lcp >= i) of the dims that can be
// a pair's lowest colliding dim, in four lists of job_cap / 4 entries each,
// by size: list 0 more than 32 members (a CTA each, count counts[0]),
// list 1 9..32 (a warp each, counts[2]), list 2 5..8 (8 lanes each,
// counts[3]), list 3 2..4 (4 lanes each, counts[4]); counts[1] = the
// largest bucket.
__global__ void k_bucket_jobs(const uint8_t* __restrict__ lcp, Seg sg, int segs, int i, int d,
                              BucketJob* __restrict__ jobs, uint64_t job_cap,
                              unsigned long long* __restrict__ counts) {
  // grid: x over the positions of a segment, y over the segments
  __shared__ uint32_t wcnt[32][4];
  __shared__ unsigned long long bbase[4];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
  const uint64_t quarter = job_cap / 4;
  const unsigned lt = (1u << lane) - 1u;
  const uint32_t seg = blockIdx.y;
  const int f = int(seg % uint32_t(sg.D));
  if (f > sg.D - d) return;                        // block-uniform: f cannot be a lowest dim
  const uint8_t* L = lcp + sg.base(int(seg));
  for (int64_t q0 = blockIdx.x * int64_t(blockDim.x); q0 < sg.M; q0 += int64_t(gridDim.x) * blockDim.x) {
    const int64_t q = q0 + threadIdx.x;
    bool emit = false;
    uint32_t n = 0, p = 0;
    if (q < sg.M) {
      p = uint32_t(q);
      if (int(L[p]) < i && int64_t(p) + 1 < sg.M && int(L[p + 1]) >= i) {
        // walk to the end of the run, eight prefix lengths at a time where
        // aligned: every byte of a word is >= i iff byte + 128 - i has its
        // top bit set (bytes are 0..8, so no carry crosses a byte)
        const uint64_t add = 0x0101010101010101ull * uint64_t(128 - i);
        int64_t e = p + 1;
        while (e + 1 < sg.M) {
          const int64_t q = e + 1;
          if ((reinterpret_cast<uintptr_t>(L + q) & 7) == 0 && q + 8 <= sg.M) {
            const uint64_t w8 = *reinterpret_cast<const uint64_t*>(L + q);
            if (((w8 + add) & 0x8080808080808080ull) == 0x8080808080808080ull) {
              e += 8;
              continue;
            }
          }
          if (int(L[q]) < i) break;
          ++e;
        }
        n = uint32_t(e - p + 1);
        emit = true;
      }
    }
    const int cls = !emit ? -1 : (n > 32u ? 0 : (n > 8u ? 1 : (n > 4u ? 2 : 3)));
    if (emit && cls == 0) atomicMax(&counts[1], (unsigned long long)n);
    // room in the four lists: one global atomic per list and block
    unsigned m[4];
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      m[c] = __ballot_sync(0xffffffffu, cls == c);
      if (lane == 0) wcnt[warp][c] = __popc(m[c]);
    }
    __syncthreads();
    if (threadIdx.x < 4) {
      const int c = threadIdx.x;
      uint32_t run = 0;
      for (int ww = 0; ww < nwarp; ++ww) {
        const uint32_t x = wcnt[ww][c];
        wcnt[ww][c] = run;
        run += x;
      }
      bbase[c] = run ? atomicAdd(&counts[c == 0 ? 0 : c + 1], (unsigned long long)run) : 0ull;
    }
    __syncthreads();
    if (cls >= 0) {
      const unsigned long long pos = bbase[cls] + wcnt[warp][cls] + __popc(m[cls] & lt);
      if (pos < quarter) jobs[cls * quarter + pos] = BucketJob{seg, p, n, 0u};
    }
    __syncthreads();                               // wcnt / bbase reused by the next iteration
  }
}

struct SubArgs {
  const uint32_t* order;
  const uint64_t* keys;
  Seg sg;
  int K, d, excl;
  HashSet hs;
  Event* events;
  uint64_t ev_cap;
  unsigned long long* counters;
  const BucketJob* jobs;
  const unsigned long long* counts;
  int cap;
  uint64_t job_cap;
};

// Byte planes 0..NQ-1 of a window's D keys (plane h, word c: byte e =
// hash value h of dim 8c + e), each key loaded once.
template <int NQ, int NW>
__device__ __forceinline__ void key_planes(const uint64_t* kw, int D, int K, uint64_t (&pl)[NQ][NW]) {
#pragma unroll
  for (int c = 0; c < NW; ++c) {
    uint64_t key[8];
#pragma unroll
    for (int e = 0; e < 8; ++e) key[e] = 8 * c + e < D ? kw[8 * c + e] : 0ull;
#pragma unroll
    for (int h = 0; h < NQ; ++h) {
      uint64_t a = 0;
#pragma unroll
      for (int e = 0; e < 8; ++e) a |= ((key[e] >> (56 - 8 * h)) & 0xFFull) << (8 * e);
      pl[h][c] = h < K ? a : 0ull;
    }
  }
}

// CTA per large bucket of prefix length I (the first I hash values equal
// in its dim f).  NW byte-plane words per hash value (dims 8c .. 8c+7 in
// word c), planes of hash values 0..I (value I only for the level
// de-duplication).  A pair is handled from its two lowest colliding dims
// (f, f2): members are split into sub-buckets by a hash of f2's first I
// values, and only pairs inside a sub-bucket are compared.
template <int NW, int I>
__global__ void __launch_bounds__(256) k_subbucket(SubArgs g) {
  constexpr int NQ = I + 1;
  extern __shared__ uint64_t sub_smem[];
  const int cap = g.cap;
  uint64_t* pl = sub_smem;                 // [NQ][NW][cap]
  uint32_t* widx = reinterpret_cast<uint32_t*>(pl + NQ * NW * cap);
  uint32_t* hist = widx + cap;
  uint32_t* bend = hist + 256;
  uint16_t* perm = reinterpret_cast<uint16_t*>(bend + 256);
  uint8_t* skey = reinterpret_cast<uint8_t*>(perm + cap);
  const int tid = threadIdx.x, lane = tid & 31;
  const int D = g.sg.D;
  const bool lvl_dup = g.K > I;
  uint64_t valid[NW];
#pragma unroll
  for (int c = 0; c < NW; ++c) {
    const int nd = D - 8 * c;
    valid[c] = nd >= 8 ? 0x8080808080808080ull
                       : (nd <= 0 ? 0ull : (0x8080808080808080ull & ((1ull << (8 * nd)) - 1)));
  }
  uint64_t njobs = g.counts[0];
  if (njobs > g.job_cap / 4) njobs = g.job_cap / 4;
  unsigned long long checks = 0;                   // pairs compared by this thread
  for (uint64_t jb = blockIdx.x; jb < njobs; jb += gridDim.x) {
    const BucketJob job = g.jobs[jb];
    const int n = int(job.n);
    if (n > cap) continue;                         // never launched with such buckets
    const int seg = int(job.seg);
    const int j = g.sg.j0 + seg / D, f = seg - (seg / D) * D;
    const uint32_t* O = g.order + g.sg.base(seg) + job.start;
    const uint64_t* Kj = g.keys + int64_t(j) * g.sg.M * D;
    __syncthreads();
    for (int q = tid; q < n; q += blockDim.x) {
      const uint32_t wv = O[q];
      widx[q] = wv;
      uint64_t kp[NQ][NW];
      key_planes<NQ, NW>(Kj + int64_t(wv) * D, D, g.K, kp);
#pragma unroll
      for (int h = 0; h < NQ; ++h)
#pragma unroll
        for (int c = 0; c < NW; ++c) pl[(h * NW + c) * cap + q] = kp[h][c];
    }
    __syncthreads();
    // second-lowest colliding dim f2 leaves d - 2 dims above it
    for (int f2 = f + 1; f2 <= D - g.d + 1; ++f2) {
      for (int b = tid; b < 256; b += blockDim.x) hist[b] = 0;
      __syncthreads();
      const int c2 = f2 >> 3, e2 = f2 & 7;
      for (int q = tid; q < n; q += blockDim.x) {
        uint32_t k = 0;
#pragma unroll
        for (int h = 0; h < I; ++h) k ^= uint32_t(pl[(h * NW + c2) * cap + q] >> (8 * e2)) << h;
        k &= 255u;
        skey[q] = uint8_t(k);
        atomicAdd(&hist[k], 1u);
      }
      __syncthreads();
      if (tid < 32) {                              // exclusive scan of 256 counts by one warp
        uint32_t v[8], run = 0;
#pragma unroll
        for (int r = 0; r < 8; ++r) { v[r] = hist[tid * 8 + r]; run += v[r]; }
        uint32_t incl = run;
        for (int o = 1; o < 32; o <<= 1) {
          uint32_t u = __shfl_up_sync(0xffffffffu, incl, o);
          if (tid >= o) incl += u;
        }
        uint32_t base = incl - run;
#pragma unroll
        for (int r = 0; r < 8; ++r) { hist[tid * 8 + r] = base; base += v[r]; }
      }
      __syncthreads();
      for (int q = tid; q < n; q += blockDim.x) {
        const uint32_t pos = atomicAdd(&hist[skey[q]], 1u);
        perm[pos] = uint16_t(q);
      }
      __syncthreads();
      for (int b = tid; b < 256; b += blockDim.x) bend[b] = hist[b];
      __syncthreads();
      // pairs inside a sub-bucket may collide in f and f2;
      // below[c]: bytes of dims < f2 in word c, only_f[c]: the byte of f
      uint64_t below[NW], only_f[NW];
#pragma unroll
      for (int c = 0; c < NW; ++c) {
        const uint64_t all = c < c2 ? ~0ull : (c == c2 ? ((1ull << (8 * e2)) - 1) : 0ull);
        below[c] = all & valid[c];
        only_f[c] = (f >> 3) == c ? (0x80ull << (8 * (f & 7))) : 0ull;
      }
      for (int r = tid; r < n; r += blockDim.x) {
        const int u = perm[r];
        const int end = int(bend[skey[u]]);
        uint64_t pu[NQ][NW];
#pragma unroll
        for (int h = 0; h < NQ; ++h)
#pragma unroll
          for (int c = 0; c < NW; ++c) pu[h][c] = pl[(h * NW + c) * cap + u];
        const uint32_t wu = widx[u];
        checks += (unsigned long long)(end > r + 1 ? end - r - 1 : 0);
        for (int r2 = r + 1; r2 < end; ++r2) {
          const int v = perm[r2];
          uint64_t m[NW];
          bool lowest = true;
          int w0 = 0;
#pragma unroll
          for (int c = 0; c < NW; ++c) {
            uint64_t x = valid[c];
#pragma unroll
            for (int h = 0; h < I; ++h) x &= zero_bytes(pu[h][c] ^ pl[(h * NW + c) * cap + v]);
            m[c] = x;
            // f and f2 are the two lowest colliding dims
            lowest = lowest && (x & below[c]) == only_f[c];
            w0 += __popcll(x);
          }
          if (!lowest || w0 < g.d) continue;
          if (lvl_dup) {
            int w1 = 0;
#pragma unroll
            for (int c = 0; c < NW; ++c)
              w1 += __popcll(m[c] & zero_bytes(pu[I][c] ^ pl[(I * NW + c) * cap + v]));
            if (w1 >= g.d) continue;
          }
          const uint32_t wv = widx[v];
          const uint32_t a = min(wu, wv), b = max(wu, wv);
          if (int64_t(b) - int64_t(a) <= g.excl) continue;
          const uint64_t key = (uint64_t(a) << 32) | b;
          if (set_contains(g.hs, key)) continue;
          const unsigned act = __activemask();
          const int leader = __ffs(act) - 1;
          unsigned long long base = 0;
          if (lane == leader) base = atomicAdd(&g.counters[0], (unsigned long long)__popc(act));
          base = __shfl_sync(act, base, leader);
          const unsigned long long pos = base + __popc(act & ((1u << lane) - 1u));
          if (pos < g.ev_cap) g.events[pos] = Event{a, b, int32_t(j), 0u};
        }
      }
      __syncthreads();
    }
  }
  for (int o = 16; o > 0; o >>= 1) checks += __shfl_xor_sync(0xffffffffu, checks, o);
  if (lane == 0 && checks) atomicAdd(&g.counters[5], checks);
}

// W lanes per small bucket (at most W members, one per lane; 32 / W
// buckets per warp): every pair is compared directly and handled from its
// lowest colliding dim f.  list = the job list (1..3) of buckets of this size.
template <int NW, int I, int W>
__global__ void __launch_bounds__(256) k_subwarp(SubArgs g, int list) {
  constexpr int NQ = I + 1;
  constexpr int J = 32 / W;                       // buckets per warp
  const int lane = threadIdx.x & 31, sub = lane / W, sl = lane % W;
  const int D = g.sg.D;
  const bool lvl_dup = g.K > I;
  uint64_t valid[NW];
#pragma unroll
  for (int c = 0; c < NW; ++c) {
    const int nd = D - 8 * c;
    valid[c] = nd >= 8 ? 0x8080808080808080ull
                       : (nd <= 0 ? 0ull : (0x8080808080808080ull & ((1ull << (8 * nd)) - 1)));
  }
  const uint64_t quarter = g.job_cap / 4;
  uint64_t njobs = g.counts[list + 1];
  if (njobs > quarter) njobs = quarter;
  const BucketJob* jl = g.jobs + uint64_t(list) * quarter;
  const uint64_t nwarps = uint64_t(gridDim.x) * (blockDim.x >> 5);
  const uint64_t wg = (blockIdx.x * uint64_t(blockDim.x) + threadIdx.x) >> 5;
  unsigned long long checks = 0;
  for (uint64_t jb0 = wg * J; jb0 < njobs; jb0 += nwarps * J) {   // warp-uniform
    const uint64_t jb = jb0 + sub;
    int n = 0, j = 0, f = 0;
    uint32_t wu = 0;
    uint64_t pu[NQ][NW];
#pragma unroll
    for (int h = 0; h < NQ; ++h)
#pragma unroll
      for (int c = 0; c < NW; ++c) pu[h][c] = 0ull;
    if (jb < njobs) {
      const BucketJob job = jl[jb];
      n = int(job.n);
      const int seg = int(job.seg);
      j = g.sg.j0 + seg / D;
      f = seg - (seg / D) * D;
      if (sl < n) {
        wu = g.order[g.sg.base(seg) + job.start + sl];
        key_planes<NQ, NW>(g.keys + (int64_t(j) * g.sg.M + wu) * D, D, g.K, pu);
      }
    }
    // dims below f must not collide: bytes of dims < f
    uint64_t below[NW];
#pragma unroll
    for (int c = 0; c < NW; ++c) {
      const int cf = f >> 3, ef = f & 7;
      below[c] = (c < cf ? ~0ull : (c == cf ? ((1ull << (8 * ef)) - 1) : 0ull)) & valid[c];
    }
    int nmax = n;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) nmax = max(nmax, __shfl_xor_sync(0xffffffffu, nmax, o));
    for (int v = 0; v < nmax - 1; ++v) {
      uint64_t pv[NQ][NW];
#pragma unroll
      for (int h = 0; h < NQ; ++h)
#pragma unroll
        for (int c = 0; c < NW; ++c) pv[h][c] = __shfl_sync(0xffffffffu, pu[h][c], v, W);
      const uint32_t wv = __shfl_sync(0xffffffffu, wu, v, W);
      bool emit = sl > v && sl < n;
      checks += emit ? 1u : 0u;
      int w0 = 0, w1 = 0;
      bool low = false;
#pragma unroll
      for (int c = 0; c < NW; ++c) {
        uint64_t x = valid[c];
#pragma unroll
        for (int h = 0; h < I; ++h) x &= zero_bytes(pu[h][c] ^ pv[h][c]);
        low = low || (x & below[c]) != 0;
        w0 += __popcll(x);
        if (lvl_dup) w1 += __popcll(x & zero_bytes(pu[I][c] ^ pv[I][c]));
      }
      emit = emit && !low && w0 >= g.d && !(lvl_dup && w1 >= g.d);
      const uint32_t a = min(wu, wv), b = max(wu, wv);
      emit = emit && int64_t(b) - int64_t(a) > g.excl;
      const uint64_t key = (uint64_t(a) << 32) | b;
      if (emit) emit = !set_contains(g.hs, key);
      const unsigned m = __ballot_sync(0xffffffffu, emit);
      if (!m) continue;
      unsigned long long base = 0;
      if (lane == __ffs(m) - 1) base = atomicAdd(&g.counters[0], (unsigned long long)__popc(m));
      base = __shfl_sync(0xffffffffu, base, __ffs(m) - 1);
      if (emit) {
        const unsigned long long pos = base + __popc(m & ((1u << lane) - 1u));
        if (pos < g.ev_cap) g.events[pos] = Event{a, b, int32_t(j), 0u};
      }
    }
  }
  for (int o = 16; o > 0; o >>= 1) checks += __shfl_xor_sync(0xffffffffu, checks, o);
  if (lane == 0 && checks) atomicAdd(&g.counters[5], checks);
}

__global__ void k_hs_clear(uint64_t* __restrict__ keys, uint64_t cap) {
  for (uint64_t q = blockIdx.x * uint64_t(blockDim.x) + threadIdx.x; q < cap;
       q += uint64_t(gridDim.x) * blockDim.x)
    keys[q] = kEmpty;
}

}  // namespace

template <bool PLAIN, int I>
static cudaError_t run_collide(const CollideArgs& g, size_t smem, cudaStream_t s) {
  cudaError_t e = allow_smem(reinterpret_cast<const void*>(k_collide<PLAIN, I>), smem);
  if (e != cudaSuccess) return e;
  MOMENTI_LAUNCH("collide", s, k_collide<PLAIN, I><<<sm_count() * 8, 128, smem, s>>>(g));
  return cudaGetLastError();
}

template <bool PLAIN>
static cudaError_t dispatch_plain(int i, const CollideArgs& g, size_t smem, cudaStream_t s) {
  switch (i) {
    case 1: return run_collide<PLAIN, 1>(g, smem, s);
    case 2: return run_collide<PLAIN, 2>(g, smem, s);
    case 3: return run_collide<PLAIN, 3>(g, smem, s);
    case 4: return run_collide<PLAIN, 4>(g, smem, s);
    case 5: return run_collide<PLAIN, 5>(g, smem, s);
    case 6: return run_collide<PLAIN, 6>(g, smem, s);
    case 7: return run_collide<PLAIN, 7>(g, smem, s);
    case 8: return run_collide<PLAIN, 8>(g, smem, s);
  }
  return cudaErrorInvalidValue;
}

static cudaError_t dispatch_collide(int i, bool plain, const CollideArgs& g, size_t smem, cudaStream_t s) {
  return plain ? dispatch_plain<true>(i, g, smem, s) : dispatch_plain<false>(i, g, smem, s);
}

cudaError_t launch_bucket_jobs(const Index& ix, int i, int j0, int j1, int d, BucketJob* jobs,
                               uint64_t job_cap, unsigned long long* counts, cudaStream_t s) {
  const int segs = (j1 - j0) * ix.D;
  Seg sg{ix.M, ix.D, j0, int((ix.M + 31) / 32)};
  int64_t gx = (ix.M + 255) / 256;
  const int64_t per_seg = std::max<int64_t>(1, (sm_count() * 16 + segs - 1) / segs);
  if (gx > per_seg) gx = per_seg;
  dim3 grid{unsigned(gx), unsigned(segs), 1u};
  MOMENTI_LAUNCH("bucket_jobs", s, k_bucket_jobs<<<grid, 256, 0, s>>>(ix.lcp, sg, segs, i, d, jobs, job_cap, counts));
  return cudaGetLastError();
}

size_t subbucket_smem(int cap, int D, int i) {
  const int nw = (D + 7) / 8;
  return size_t(cap) * (8 * nw * (i + 1) + 4 + 2 + 1) + 2 * 256 * 4 + 16;
}

int subbucket_cap(int D, int i) {
  for (int cap = 8192; cap >= 1024; cap /= 2)
    if (subbucket_smem(cap, D, i) <= size_t(200) * 1024) return cap;
  return 0;
}

template <int NW, int I>
static cudaError_t run_subbucket(const SubArgs& g, size_t smem, cudaStream_t s) {
  cudaError_t e = allow_smem(reinterpret_cast<const void*>(k_subbucket<NW, I>), smem);
  if (e != cudaSuccess) return e;
  int per_sm = int((size_t(200) * 1024) / smem);
  if (per_sm < 1) per_sm = 1;
  if (per_sm > 8) per_sm = 8;
  MOMENTI_LAUNCH("subbucket", s, k_subbucket<NW, I><<<sm_count() * per_sm, 256, smem, s>>>(g));
  MOMENTI_LAUNCH("subwarp", s, k_subwarp<NW, I, 32><<<sm_count() * 8, 256, 0, s>>>(g, 1));
  MOMENTI_LAUNCH("subwarp", s, k_subwarp<NW, I, 8><<<sm_count() * 8, 256, 0, s>>>(g, 2));
  MOMENTI_LAUNCH("subwarp", s, k_subwarp<NW, I, 4><<<sm_count() * 8, 256, 0, s>>>(g, 3));
  return cudaGetLastError();
}

cudaError_t launch_subbucket(const Index& ix, int i, int j0, int j1, int d, const HashSet& hs,
                             const CollideScratch& cs, const BucketJob* jobs, uint64_t job_cap,
                             const unsigned long long* counts, int max_bucket, cudaStream_t s) {
  if (ix.D > 16 || i < 1 || i > 3 || max_bucket > subbucket_cap(ix.D, i)) return cudaErrorInvalidValue;
  Seg sg{ix.M, ix.D, j0, int((ix.M + 31) / 32)};
  const int cap = std::max(256, ((max_bucket + 255) / 256) * 256);
  SubArgs g{ix.order, ix.keys, sg, ix.K, d, ix.excl, hs, cs.events, cs.ev_cap, cs.counters, jobs,
            counts, cap, job_cap};
  const size_t smem = subbucket_smem(cap, ix.D, i);
  const bool two = ix.D > 8;
  switch (i) {
    case 1: return two ? run_subbucket<2, 1>(g, smem, s) : run_subbucket<1, 1>(g, smem, s);
    case 2: return two ? run_subbucket<2, 2>(g, smem, s) : run_subbucket<1, 2>(g, smem, s);
    default: return two ? run_subbucket<2, 3>(g, smem, s) : run_subbucket<1, 3>(g, smem, s);
  }
}

cudaError_t launch_hashset_clear(const HashSet& hs, cudaStream_t s) {
  MOMENTI_LAUNCH("hs_clear", s, k_hs_clear<<<sm_count() * 8, 256, 0, s>>>(hs.keys, hs.cap));
  return cudaGetLastError();
}

cudaError_t launch_collide(const Index& ix, int i, int j0, int j1, int d, const HashSet& hs,
                           const CollideScratch& cs, int mode_plain, uint64_t* out_pairs,
                           uint64_t out_cap, cudaStream_t s) {
  const int segs = (j1 - j0) * ix.D;
  const int64_t C = (ix.M + 31) / 32;
  if (segs > cs.seg_cap || C > cs.chunk_cap) return cudaErrorInvalidValue;
  Seg sg{ix.M, ix.D, j0, int(C)};
  const int64_t E = int64_t(segs) * C;
  uint64_t* toff = cs.ntile;
  MOMENTI_LAUNCH("chunk_agg", s, k_chunk_agg<<<unsigned((E * 32 + 255) / 256), 256, 0, s>>>(ix.lcp, sg, segs, i, d, cs.cagg, toff));
  MOMENTI_LAUNCH("chunk_scan", s, k_chunk_scan<<<segs, 1024, 0, s>>>(ix.lcp, sg, i, cs.cagg, cs.cbs, toff));
  const int64_t nb = (E + kScanBlock - 1) / kScanBlock;
  uint64_t* bsum = cs.scan_tmp;
  MOMENTI_LAUNCH("scan_local", s, k_scan_local<<<unsigned(nb), kScanBlock, 0, s>>>(toff, E, bsum));
  MOMENTI_LAUNCH("scan_top", s, k_scan_top<<<1, kScanBlock, 0, s>>>(bsum, nb, toff + E));
  MOMENTI_LAUNCH("scan_add", s, k_scan_add<<<unsigned(nb), kScanBlock, 0, s>>>(toff, E, bsum));
  CollideArgs g{ix.order, ix.lcp, ix.keys, sg, segs, i, ix.K, d, ix.excl, cs.cbs, toff, hs,
                cs.events, cs.ev_cap, cs.counters, out_pairs, out_cap};
  const int G = (ix.D + 7) / 8;
  const int NP = (!mode_plain && i < ix.K) ? i + 1 : i;
  size_t smem = size_t(4) * (64 * G * NP + 32) * sizeof(uint64_t);
  cudaError_t e = dispatch_collide(i, mode_plain != 0, g, smem, s);
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}

}  // namespace momenti

