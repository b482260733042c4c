// Internal declarations shared by the kernel translation units and the
// host orchestration of the motif search.  Not part of the public ABI.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>
#include <cuda_fp16.h>

#include <vector>

namespace momenti {

// Window count limit: the index sort puts tiles of 2048 windows on the
// grid's y dimension (at most 65535 blocks), which is tighter than the
// 32-bit window index.
constexpr int64_t kMaxWindows = int64_t(65535) * 2048;
constexpr int kKeyBytes = 8;          // one byte per concatenated hash value
constexpr int kRepStride = 8;         // projections per repetition in the layouts
constexpr double kFlatRel = 1e-8;     // flat window: sigma <= kFlatRel (1 + |mu|)

// Device-resident series, window statistics, hash functions and index.
struct Index {
  int64_t n = 0, M = 0;
  int D = 0, w = 0, K = 0, L = 0, Wp = 0, excl = 0;
  double r = 0.0;
  float inv_r = 0.f;
  bool has_lo = false;
  float* xs_hi = nullptr;     // [D][n]  series, float32 part
  float* xs_lo = nullptr;     // [D][n]  float64 input only: x - double(hi), as float
  float* xT = nullptr;        // [n][Dp] point-major copy of xs_hi (D <= 8), dims padded with 0
  float* xlT = nullptr;       // [n][Dp] point-major copy of xs_lo
  int Dp = 0;                 // 4, 8 or 16 when xT is present
  float* xW = nullptr;        // [n][DW] point-major copy of xs_hi for 16 < D <= 64, float32 input
  int DW = 0;                 // 32 or 64 when xW is present
  float* smT = nullptr;       // [n-15][Dp] means of 16 consecutive points (D <= 8, w >= 32)
  float* stT = nullptr;       // [M][3][Dp] point-major mu_hi, mu_lo, inv_sig (D <= 8)
  float* isT = nullptr;       // [M][Dp] 1/sigma (padding dims 1), float32 input, D <= 16
  float* isW = nullptr;       // [M][DW] 1/sigma (padding dims 1), with xW
  uint8_t* cflag = nullptr;   // [M] column window not testable in float32 by the sweep
  double* mu = nullptr;       // [D][M]
  double* sig = nullptr;      // [D][M]
  float* mu_hi = nullptr;     // [D][M]  float(mu)
  float* mu_lo = nullptr;     // [D][M]  float(mu - double(mu_hi))
  float* inv_sig = nullptr;   // [D][M]  1/sigma, 0 for flat windows
  __half* a16 = nullptr;      // [D][N][Wp]   N = L * 8, K-major rows for tensor cores
  float* a32 = nullptr;       // [D][Wp][N]   same values, float32, for CUDA cores
  float* boff = nullptr;      // [D][N]       b = u * r
  uint64_t* keys = nullptr;   // [L][M][D]
  uint32_t* order = nullptr;  // [L][D][M]
  uint8_t* lcp = nullptr;     // [L][D][M]
};

// One verified pair as it travels to the host.
struct PairRec {
  uint32_t a, b;      // a < b
  int32_t j;          // 0-based repetition of first collision in the chunk
  float dist_d;       // sum of the d smallest per-dimension distances
  float dist_max;     // largest distance among the d selected dimensions
  uint32_t pad;
  uint64_t dims;      // mask of the d selected dimensions
};
static_assert(sizeof(PairRec) == 32, "PairRec layout");

// ---- profile.cu ---------------------------------------------------------
// Every launch is bracketed by prof_begin / prof_end (launch counter and,
// for the selected kernel, CUDA events on the launching stream).
void prof_begin(const char* name, cudaStream_t s);
void prof_end(const char* name, cudaStream_t s);
// Opt a kernel in to `bytes` of dynamic shared memory on the current
// device.  The limit only ever rises (under a lock), so a launch on one
// thread never sees it lowered by another thread's smaller request.
cudaError_t allow_smem(const void* func, size_t bytes);
// Streaming multiprocessors of the current device (cudaDevAttrMultiProcessorCount,
// queried once per device); grids are sized in multiples of it.
int sm_count();
#define MOMENTI_LAUNCH(name, stream, ...)      \
  do {                                         \
    ::momenti::prof_begin(name, stream);       \
    __VA_ARGS__;                               \
    ::momenti::prof_end(name, stream);         \
  } while (0)

// ---- k_stats.cu ---------------------------------------------------------
cudaError_t launch_split_series(const void* src, int dtype, int64_t n, int D, int64_t ld,
                                float* hi, float* lo, cudaStream_t s);
cudaError_t launch_window_stats(const Index& ix, cudaStream_t s);
// xT / xlT from xs_hi / xs_lo, and smT (ix.Dp set)
cudaError_t launch_point_major(const Index& ix, cudaStream_t s);
// stT from the window statistics (after launch_window_stats)
cudaError_t launch_stats_point_major(const Index& ix, cudaStream_t s);
// min/max of the projections of S evenly spaced windows per dim onto the K
// vectors of repetition 0; out2 = {min, max} (device, 2 floats).
cudaError_t launch_r_sample(const Index& ix, int S, float* out2, cudaStream_t s);
// Hash functions drawn on the device (Philox4x32-10 + Box-Muller):
// a ~ N(0,1) rounded to half, u ~ U[0,1).  a_out [D][L][K][w], u_out [D][L][K].
cudaError_t launch_draw_hash(uint64_t seed, int D, int L, int K, int w, float* a_out,
                             float* u_out, cudaStream_t s);
// Lay the draws out for the projection kernels: a16/a32 padded to 8 per
// repetition and Wp columns (a rounded to half); boff = u * r (needs ix.r).
cudaError_t launch_layout_hash(const Index& ix, const float* a_src, int L_src, cudaStream_t s);
cudaError_t launch_layout_boff(const Index& ix, const float* u_src, int L_src, cudaStream_t s);

// ---- k_hash_fp32.cu -----------------------------------------------------
cudaError_t launch_proj_hash_fp32(const Index& ix, int j0, int j1, cudaStream_t s);

// ---- k_hash_tc.cu -------------------------------------------------------
// tcgen05 projection + hash for repetitions [j0, j1).  Values within 2^-11
// of a bucket boundary are appended to flags as (f << 56 | n << 32 | a);
// launch_rehash_fp32 recomputes them in the canonical FP32 form.  *err is
// raised if a bounded wait ran out.
bool tc_supported();
size_t proj_hash_tc_smem(int Wp, bool lo);
cudaError_t launch_proj_hash_tc(const Index& ix, int j0, int j1, uint64_t* flags,
                                uint32_t flag_cap, uint32_t* flag_count, int* err, cudaStream_t s);
cudaError_t launch_rehash_fp32(const Index& ix, const uint64_t* flags, const uint32_t* flag_count,
                               uint32_t flag_cap, cudaStream_t s);

// ---- k_tensor.cu --------------------------------------------------------
// Tensoring: keys [j][M][D] of repetitions [j0, j1) of L = m^2 from the keys
// half [2m][M][D] of the half functions (left l at 2 l, right r at 2 r + 1).
cudaError_t launch_tensor_keys(const Index& ix, const uint64_t* half, int m, int j0, int j1,
                               cudaStream_t s);

// ---- k_sort.cu ----------------------------------------------------------
// Largest chunk one CTA sorts in shared memory (the most-significant-digit
// partition goes one hash value deeper for larger buckets).
constexpr int kSortLocalMax = 2048;
// A range of one segment that one level partitions by one hash value.
struct SortItem {
  uint32_t seg;      // segment (repetition-major within the batch)
  uint32_t start;    // first rank of the range in its segment
  uint32_t size;
  uint32_t hist0;    // first histogram tile of the range
  uint32_t lcp0;     // hash values its first entry shares with its predecessor
  uint32_t pad[3];
};
// A range of one segment sorted completely in shared memory (or, equal keys,
// already in order).
struct SortChunk {
  uint32_t seg, start, size;
  uint8_t lcp0, buf, equal, pad;
};
struct SortCaps {
  int64_t item_cap = 0, tile_cap = 0, chunk_cap = 0;
};
struct SortScratch {
  uint64_t* k0 = nullptr; uint64_t* k1 = nullptr;   // [segs][M] ping-pong keys
  uint32_t* v0 = nullptr; uint32_t* v1 = nullptr;   // [segs][M] ping-pong windows
  uint32_t* hist = nullptr;                         // [tiles][256] digit counts / offsets
  SortItem* items[2] = {nullptr, nullptr};          // this level's and the next level's
  uint64_t* tile_item[2] = {nullptr, nullptr};      // launch tile -> (tile in item << 32 | item)
  SortChunk* chunks = nullptr;
  uint32_t* cnt = nullptr;                          // 64 device counters
  uint32_t* host_cnt = nullptr;   // pinned copy of the counters: levels sized by the host;
                                  // nullptr: every level launched with fixed grids
  SortCaps caps;
  int64_t M = 0, cap_entries = 0;
  int segs = 0;
};
constexpr int kSortTile = 2048;           // entries per partition tile
// Capacities for segs segments of M entries: items of one level (buckets
// above kSortLocalMax are disjoint), launch tiles of one level, chunks of
// all levels together (greedy packing leaves at most two chunks per
// kSortLocalMax entries, plus one per bucket boundary that a large bucket
// or an item makes).
constexpr SortCaps sort_caps(int64_t M, int segs) {
  SortCaps c;
  const int64_t entries = M * segs;
  const int64_t tpm = (M + kSortTile - 1) / kSortTile;
  const int64_t big = entries / kSortLocalMax + 1;
  c.item_cap = int64_t(segs) > big ? int64_t(segs) : big;
  const int64_t t0 = int64_t(segs) * tpm, t1 = entries / kSortTile + c.item_cap + 1;
  c.tile_cap = t0 > t1 ? t0 : t1;
  c.chunk_cap = 2 * int64_t(segs) + (2 + 2 * 8) * big + 16;
  return c;
}
constexpr size_t sort_up256(size_t b) { return (b + 255) & ~size_t(255); }
// Bytes of one region holding every scratch array for segs segments of M.
constexpr size_t sort_scratch_bytes(int64_t M, int segs) {
  const SortCaps c = sort_caps(M, segs);
  const size_t e = size_t(M) * size_t(segs);
  return 2 * sort_up256(e * 8) + 2 * sort_up256(e * 4) + sort_up256(size_t(c.tile_cap) * 256 * 4) +
         2 * sort_up256(size_t(c.item_cap) * sizeof(SortItem)) +
         2 * sort_up256(size_t(c.tile_cap) * 8) + sort_up256(size_t(c.chunk_cap) * sizeof(SortChunk)) +
         sort_up256(64 * 4);
}
// The scratch arrays laid out in one region of sort_scratch_bytes(M, segs)
// bytes (256-byte aligned); host_cnt is left null.
SortScratch sort_scratch_carve(void* base, int64_t M, int segs);
// Sort repetitions [j0, j1): all D segments of each, writing order/lcp.
cudaError_t launch_sort_reps(const Index& ix, int j0, int j1, const SortScratch& sc,
                             cudaStream_t s);

// ---- k_collide.cu -------------------------------------------------------
constexpr uint64_t kSetEmpty = ~0ull;
constexpr int kSetMaxProbe = 512;
// splitmix64 finalizer (Steele, Lea, Flood 2014): slot hash of a pair key
__device__ __forceinline__ uint64_t set_hash(uint64_t x) {
  x ^= x >> 30;
  x *= 0xbf58476d1ce4e5b9ull;
  x ^= x >> 27;
  x *= 0x94d049bb133111ebull;
  x ^= x >> 31;
  return x;
}
// Device set of close pairs verified so far (open addressing, keys only):
// a cache that spares re-verifying them; cleared by the host when half full.
struct HashSet {
  uint64_t* keys = nullptr;   // a << 32 | b, EMPTY = ~0ull
  uint64_t cap = 0;           // power of two
};
// A candidate of Algorithm 1: pair (a < b) with W >= d in repetition j.
struct Event {
  uint32_t a, b;
  int32_t j;
  uint32_t pad;
};
struct CollideScratch {
  int32_t* cagg = nullptr;     // [segs][chunks] last bucket start in chunk, or -1
  int32_t* cbs = nullptr;      // [segs][chunks] bucket start of the chunk's first rank
  uint64_t* ntile = nullptr;   // [segs*chunks + 1] tiles per chunk, then exclusive scan
  uint64_t* scan_tmp = nullptr;   // [segs*chunks / 1024 + 2]
  Event* events = nullptr;
  uint64_t ev_cap = 0;
  // [0] events (or plain pairs), [1] close records, [2] set inserts,
  // [3] events dropped by the lower bound, [4] verified pairs dropped at or
  // above the threshold, [5] pairs compared by the sub-bucket form
  unsigned long long* counters = nullptr;
  int64_t seg_cap = 0;            // segments the arrays can hold
  int64_t chunk_cap = 0;          // chunks per segment
};
// Collision counting at prefix length i for repetitions [j0, j1): every
// non-trivial pair with W >= d (handled from its first colliding dim, not
// already a candidate at length i+1 in the same repetition, not yet in the
// set) becomes an event.  mode_plain != 0: every such pair once, without
// the level and set checks, to out_pairs (a << 32 | b).
cudaError_t launch_collide(const Index& ix, int i, int j0, int j1, int d, const HashSet& hs,
                           const CollideScratch& cs, int mode_plain, uint64_t* out_pairs,
                           uint64_t out_cap, cudaStream_t s);
cudaError_t launch_hashset_clear(const HashSet& hs, cudaStream_t s);

// Prefix length 1, d >= 2, D <= 8: the buckets of the chunk as jobs
// (segment, first rank, size), then pairs found by splitting each bucket
// by the first hash value of every higher dimension (a pair with W >= 2
// collides in a second dim f2); each W >= d pair is emitted once, from its
// two lowest colliding dims.  Same events as launch_collide.
struct BucketJob {
  uint32_t seg, start, n, pad;
};
// Largest bucket (members) a CTA holds in shared memory at prefix length i.
int subbucket_cap(int D, int i);
// Buckets of prefix length i (1..3) in four lists of job_cap/4 entries by
// size: > 32 members (counts[0]), 9..32 (counts[2]), 5..8 (counts[3]),
// 2..4 (counts[4]); counts[1] = the largest bucket.  counts (5 entries)
// must be zeroed by the caller.
cudaError_t launch_bucket_jobs(const Index& ix, int i, int j0, int j1, int d, BucketJob* jobs,
                               uint64_t job_cap, unsigned long long* counts, cudaStream_t s);
// Collision counting at prefix length i (1..3, d >= 2, D <= 16) from the
// bucket jobs: a CTA per large bucket (sub-buckets by a second dim), a
// warp per small one; the same events as launch_collide.
cudaError_t launch_subbucket(const Index& ix, int i, int j0, int j1, int d, const HashSet& hs,
                             const CollideScratch& cs, const BucketJob* jobs, uint64_t job_cap,
                             const unsigned long long* counts, int max_bucket, cudaStream_t s);

// ---- k_verify.cu --------------------------------------------------------
// Verifies every event of the chunk: pairs with dist_d < tau are written to
// rec (count counters[1], may exceed rec_cap) and offered to the set.
cudaError_t launch_verify_events(const Index& ix, int d, const HashSet& hs,
                                 const CollideScratch& cs, float tau, PairRec* rec,
                                 uint64_t rec_cap, cudaStream_t s);
// Verify explicit pairs (a,b) packed as a << 32 | b; per_dim optional [m][D].
cudaError_t launch_verify_pairs(const Index& ix, int d, const uint64_t* pairs, int64_t m,
                                int fp64, double* per_dim, double* dist_d, uint64_t* dims,
                                cudaStream_t s);
// Exact all-pairs: every non-trivial pair with approximate dist_d <= tau
// appended to out (a << 32 | b) with count in *count (may exceed cap).
// Output of an all-pairs sweep: pairs whose approximate dist_d (float32
// Pearson form, within 1% + 0.01 of the exact value) lies in (lo, thr]
// go to out / out_d while count < cap; count counts them all and hist
// (kApBins bins over (lo, thr], may be NULL) their distribution.
constexpr int kApBins = 4096;
struct ApRec {
  uint64_t* out = nullptr;
  float* out_d = nullptr;
  uint64_t cap = 0;
  unsigned long long* count = nullptr;
  uint32_t* hist = nullptr;
  float lo = -1.f;
  float hscale = 0.f;          // kApBins / (thr - lo)
};
cudaError_t launch_allpairs(const Index& ix, int d, float thr, const ApRec& rc, cudaStream_t s);
// Whether the row-staged sweep of wide series (16 < D <= 64) takes this index
// (a point-major copy, and its staged rows fit a CTA's shared memory).
bool rows2_usable(const Index& ix);
// ---- k_wide64_*.cu: the 64-dimension sweeps, each instantiated in a
// translation unit of its own (they dominate the build; units compile in
// parallel).  gy_max cuts the grid to its first diagonal blocks.
cudaError_t launch_rows4_64(const Index& ix, int d, float thr, const ApRec& rc, cudaStream_t s,
                            int64_t gy_max);
cudaError_t launch_rows2_64(const Index& ix, int d, float thr, const ApRec& rc, cudaStream_t s,
                            int64_t gy_max);
cudaError_t launch_rows2_64_rowmin(const Index& ix, int d, float* rowmin, cudaStream_t s);
cudaError_t launch_wide64(const Index& ix, int d, float thr, const ApRec& rc, float* rowmin,
                          bool rowmin_mode, cudaStream_t s);

// One series' recording sweep inside a batched launch.
struct SweepJob {
  Index ix;
  ApRec rc;
  float thr = 0.f;
  int d = 0;
};
struct SweepItem {
  uint32_t job, bx, by;     // series, row block (kSeg windows), diagonal block
};
// Whether the sweep of this index can join a batched launch (float32
// input, D <= 16, the statistics form).
bool sweep_batchable(const Index& ix);
// The recording sweeps of several series (each batchable) in one
// persistent launch per padded dimension count, on stream s; every job's
// record buffers must be ready on s.
cudaError_t launch_allpairs_batch(const std::vector<SweepJob>& jobs, cudaStream_t s);
// The column table of the statistics sweep (isT, cflag), after the window
// statistics; nothing when the index has no isT.
cudaError_t launch_col_prep(const Index& ix, cudaStream_t s);
// Recorded pairs whose approximate distance lies in (lo, hi], compacted.
cudaError_t launch_select_pairs(const uint64_t* pairs, const float* dd, uint64_t m, float lo,
                                float hi, uint64_t* out, unsigned long long* count, cudaStream_t s);
// Row minima of dist_d over non-trivial partners (approximate), for the
// first threshold of the all-pairs path; rowmin [M].
cudaError_t launch_allpairs_rowmin(const Index& ix, int d, float* rowmin, cudaStream_t s);

}  // namespace momenti
