// Host side of the C ABI declared in include/momenti.h: argument checks,
// the memory planner, the hash-all pipeline (the hashing step of
// Algorithm 1 and the index of Section 4), the traversal driver with TOP and
// STOP (the prefix loop of Algorithm 1, with Algorithm 2), the exact
// all-pairs path (Algorithm 1's final fallback) and the float64
// re-verification of the result.
//
// TOP: Algorithm 1 keeps a bounded priority queue; with the trivial-match
// rule of the top-k definition (Section 3.1) one new pair can displace two
// kept ones, so TOP here is the greedy selection (ascending dist_d, then a,
// then b; a pair is taken iff both of its windows are more than eps away
// from both windows of every taken pair) over every distinct pair verified
// so far, recomputed only when a new pair lands below the current k-th.
//
// Repetitions are processed in chunks on the device; the host replays the
// chunk's new pairs in the paper's order (by repetition, as each pair is
// tagged with the first repetition in which it became a candidate) and
// evaluates STOP after each repetition, so the result and the stopping
// point are those of the sequential Algorithm 1.
#include "../../include/momenti.h"
#include "internal.h"

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <thread>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <memory>
#include <mutex>
#include <new>
#include <string>
#include <unordered_map>
#include <unordered_set>
#include <vector>

using namespace momenti;

constexpr int kChunkReps = 64;   // repetitions per device round trip of the traversal

namespace {

struct PoolEntry {
  double dd;        // dist_d
  double dmax;      // dist_d^max
  uint32_t a, b;
  uint64_t dims;
};

bool pair_less(const PoolEntry& x, const PoolEntry& y) {
  if (x.dd != y.dd) return x.dd < y.dd;
  if (x.a != y.a) return x.a < y.a;
  return x.b < y.b;
}

// Greedy top-k under the trivial-match exclusion over entries sorted by
// pair_less; returns indices of the accepted entries.
std::vector<size_t> greedy(const std::vector<PoolEntry>& sorted, int k, int64_t eps) {
  std::vector<size_t> acc;
  for (size_t q = 0; q < sorted.size() && int(acc.size()) < k; ++q) {
    const PoolEntry& c = sorted[q];
    if (int64_t(c.b) - int64_t(c.a) <= eps) continue;
    bool ok = true;
    for (size_t t : acc) {
      const PoolEntry& s = sorted[t];
      int64_t xs[2] = {c.a, c.b}, ys[2] = {s.a, s.b};
      for (int u = 0; u < 2 && ok; ++u)
        for (int v = 0; v < 2 && ok; ++v)
          if (std::llabs(xs[u] - ys[v]) <= eps) ok = false;
      if (!ok) break;
    }
    if (ok) acc.push_back(q);
  }
  return acc;
}

double std_normal_cdf(double x) { return 0.5 * std::erfc(-x / std::sqrt(2.0)); }

// Eq. (eucl-collision-probability).
double collision_probability(double R, double r) {
  if (R <= 0.0) return 1.0;
  const double c = r / R;
  return 1.0 - 2.0 * std_normal_cdf(-c) -
         2.0 / (std::sqrt(2.0 * M_PI) * c) * (1.0 - std::exp(-c * c / 2.0));
}

// Lemma stop (Eq. probnotcolliding) / Algorithm 2; i, j 1-based.
double failure_bound(double dist_max, int i, int j, int K, int L, int d, double r) {
  const double p = std::pow(collision_probability(dist_max, r), d);
  const double first = std::pow(1.0 - std::pow(p, i), j);
  if (i == K) return first;
  return first * std::pow(1.0 - std::pow(p, i + 1), L - j);
}

// Open-addressing set of pair keys (host).
struct KeySet {
  std::vector<uint64_t> slot;
  size_t used = 0;
  static constexpr uint64_t kEmpty = ~0ull;
  static uint64_t mix(uint64_t x) {
    x ^= x >> 30; x *= 0xbf58476d1ce4e5b9ull; x ^= x >> 27; x *= 0x94d049bb133111ebull;
    return x ^ (x >> 31);
  }
  bool insert(uint64_t key) {   // true if new
    if ((used + 1) * 2 > slot.size()) grow();
    size_t m = slot.size() - 1, h = size_t(mix(key)) & m;
    while (slot[h] != kEmpty) {
      if (slot[h] == key) return false;
      h = (h + 1) & m;
    }
    slot[h] = key;
    ++used;
    return true;
  }
  void grow() {
    std::vector<uint64_t> old;
    old.swap(slot);
    slot.assign(std::max<size_t>(1 << 16, old.size() * 2), kEmpty);
    used = 0;
    for (uint64_t k : old)
      if (k != kEmpty) insert(k);
  }
};

struct Pool {
  std::vector<PoolEntry> items;   // items[0, sorted) sorted by pair_less, the rest appended
  size_t sorted = 0;
  KeySet seen;
  std::vector<PoolEntry> top;     // current greedy selection
  double tau_trunc = INFINITY;    // every pair with dist_d < tau_trunc is held
  size_t cap = size_t(1) << 22;
  int k = 1;
  int64_t eps = 0;

  double kth() const { return int(top.size()) == k ? top.back().dd : INFINITY; }
  bool valid() const { return int(top.size()) == k && top.back().dd < tau_trunc; }

  void sort_all() {
    if (sorted < items.size()) {
      std::sort(items.begin() + sorted, items.end(), pair_less);
      std::inplace_merge(items.begin(), items.begin() + sorted, items.end(), pair_less);
      sorted = items.size();
    }
  }

  // a new pair not after the k-th changes the selection only if no taken
  // pair that precedes it is within eps of one of its windows
  bool changes_top(const PoolEntry& c) const {
    if (int(top.size()) < k) return true;
    if (!pair_less(c, top.back())) return false;
    if (int64_t(c.b) - int64_t(c.a) <= eps) return false;
    for (const PoolEntry& t : top) {
      if (!pair_less(t, c)) break;
      const int64_t xs[2] = {c.a, c.b}, ys[2] = {t.a, t.b};
      for (int u = 0; u < 2; ++u)
        for (int v = 0; v < 2; ++v)
          if (std::llabs(xs[u] - ys[v]) <= eps) return false;
    }
    return true;
  }

  void add(const PairRec* r, size_t m) {
    bool dirty = false;
    for (size_t q = 0; q < m; ++q) {
      if (double(r[q].dist_d) >= tau_trunc) continue;
      const uint64_t key = (uint64_t(r[q].a) << 32) | r[q].b;
      if (!seen.insert(key)) continue;
      PoolEntry c{double(r[q].dist_d), double(r[q].dist_max), r[q].a, r[q].b, r[q].dims};
      if (!dirty && changes_top(c)) dirty = true;
      items.push_back(c);
    }
    if (items.size() > cap) {
      sort_all();
      const size_t keep = cap / 2;
      tau_trunc = std::min(tau_trunc, items[keep].dd);
      items.resize(keep);
      sorted = keep;
      dirty = true;
    }
    if (dirty) {
      sort_all();
      auto acc = greedy(items, k, eps);
      top.clear();
      for (size_t q : acc) top.push_back(items[q]);
    }
  }
};

struct DevBuf {
  void* p = nullptr;
  size_t bytes = 0;
};

// TOP and stopping state of one dimensionality d.
struct DState {
  int d = 0;
  Pool pool;
  bool done = false;
  int stop_i = 0, stop_j = 0;
  double fb = 1.0;
  float tau = INFINITY;       // verified pairs at or above it cannot enter this TOP
};

// A traversal in progress (the anytime search): one state per d, and the
// cursor (level i, next repetition j0) where the next chunk starts.
struct SearchState {
  int d_low = 0, d_high = 0;
  std::vector<DState> ds;
  int i = 0, j0 = 0, d_cur = 0;
  int last_i = 0, last_j = 0;     // the last repetition processed (1-based j), 0 0 before any
  int switch_level = 0;
  double prev_rep_ms = 0.0;       // predicted cost of one repetition at the previous level's probe
  bool ended = false;             // STOP for every d, the cost switch, or the loop's end
  momenti_stats st{};
};

}  // namespace

// The batching form's sweep service.  The workers of momenti_topk_batch
// hand it the recording sweeps of their exact paths (batchable indexes:
// float32, D <= 16).  Once every worker still running is waiting here, or
// the oldest request has waited 2 ms, the pending sweeps run together in
// one persistent launch on the service's stream, ordered after what each
// requester queued on its own stream and before its next work there.
class SweepBatcher {
 public:
  explicit SweepBatcher(int workers) : active_(workers) {}
  ~SweepBatcher() {
    if (stream_) cudaStreamDestroy(stream_);
  }
  SweepBatcher(const SweepBatcher&) = delete;
  SweepBatcher& operator=(const SweepBatcher&) = delete;

  cudaError_t sweep(const Index& ix, int d, float thr, const ApRec& rc, cudaStream_t s) {
    Req r;
    r.job.ix = ix;
    r.job.rc = rc;
    r.job.thr = thr;
    r.job.d = d;
    r.s = s;
    std::unique_lock<std::mutex> lk(mu_);
    pending_.push_back(&r);
    const auto t0 = std::chrono::steady_clock::now();
    cv_.notify_all();
    while (!r.done) {
      const bool all_waiting = int(pending_.size()) >= active_;
      const bool waited = std::chrono::steady_clock::now() - t0 > std::chrono::milliseconds(2);
      if (!flushing_ && !pending_.empty() && (all_waiting || waited)) {
        flush(lk);
        continue;
      }
      cv_.wait_for(lk, std::chrono::microseconds(500));
    }
    return r.err;
  }

  // A worker has no more series.
  void worker_done() {
    std::lock_guard<std::mutex> lk(mu_);
    --active_;
    cv_.notify_all();
  }

  uint64_t launches() const { return launches_; }

 private:
  struct Req {
    SweepJob job;
    cudaStream_t s = nullptr;
    bool done = false;
    cudaError_t err = cudaSuccess;
  };

  void flush(std::unique_lock<std::mutex>& lk) {
    std::vector<Req*> batch;
    batch.swap(pending_);
    flushing_ = true;
    lk.unlock();
    cudaError_t e = cudaSuccess;
    cudaEvent_t ev = nullptr;
    // every request of the batch is answered, whatever happens here (a
    // host allocation that fails reports an error to each requester)
    try {
      if (!stream_) e = cudaStreamCreateWithFlags(&stream_, cudaStreamNonBlocking);
      if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
      std::vector<SweepJob> jobs;
      for (Req* q : batch) {
        if (e != cudaSuccess) break;
        // the batch waits for the requester's queued work (counters, buffers)
        e = cudaEventRecord(ev, q->s);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(stream_, ev, 0);
        jobs.push_back(q->job);
      }
      if (e == cudaSuccess) e = launch_allpairs_batch(jobs, stream_);
      // each requester's next work follows the launch
      if (e == cudaSuccess) e = cudaEventRecord(ev, stream_);
      for (Req* q : batch)
        if (e == cudaSuccess) e = cudaStreamWaitEvent(q->s, ev, 0);
      if (e == cudaSuccess) e = cudaStreamSynchronize(stream_);
    } catch (...) {
      if (stream_) cudaStreamSynchronize(stream_);
      e = cudaErrorMemoryAllocation;
    }
    if (ev) cudaEventDestroy(ev);
    lk.lock();
    ++launches_;
    for (Req* q : batch) {
      q->err = e;
      q->done = true;
    }
    flushing_ = false;
    cv_.notify_all();
  }

  std::mutex mu_;
  std::condition_variable cv_;
  int active_;
  bool flushing_ = false;
  std::vector<Req*> pending_;
  cudaStream_t stream_ = nullptr;
  uint64_t launches_ = 0;
};

struct momenti_handle {
  momenti_params p{};
  std::string err;
  cudaStream_t stream = nullptr;
  std::vector<float> user_a, user_u;
  int user_D = 0, user_L = 0, user_K = 0;
  Index ix;
  bool ready = false;
  std::vector<DevBuf> bufs;
  uint64_t device_bytes = 0;
  SortScratch sort;
  CollideScratch cs;
  HashSet hs;
  PairRec* rec_dev = nullptr;
  PairRec* rec_host = nullptr;
  uint64_t rec_cap = 0;
  uint64_t set_fill = 0;
  uint64_t ev_budget = uint64_t(1) << 30;
  BucketJob* jobs = nullptr;                // prefix-length-1 bucket jobs
  uint64_t job_cap = 0;
  unsigned long long* job_counts = nullptr;
  unsigned long long* cnt_host = nullptr;
  uint32_t* sort_cnt_host = nullptr;        // pinned copy of the index sort's level counters
  int chunk_reps = 32;
  double t_hash_ms = 0, t_sort_ms = 0;
  bool used_tc = false;
  uint64_t n_flagged = 0;
  int sort_reps = 1;
  uint64_t hp_gen = 0, built_gen = ~0ull;   // hash-parameter generations
  float* draw_a = nullptr;                  // device copies of the hash draws
  float* draw_u = nullptr;
  uint64_t* flags = nullptr;                // near-boundary list of the tensor-core form
  uint32_t flag_cap = 0;
  uint32_t* small = nullptr;                // r min/max, flag count, error flag
  cudaStream_t own_stream = nullptr;        // created for the batching form
  momenti_params built_p{};                 // parameters the index was built with
  size_t rec_host_cap = 0;                  // pinned record buffer (kept across rebuilds)
  std::unique_ptr<SearchState> search;      // the traversal in progress, if any
  SweepBatcher* batcher = nullptr;          // the batching form's sweep service, if any
};

namespace {

// Records the message of a failing call (never throws: a message that
// cannot be stored is dropped, the code still reports the failure).
int fail(momenti_handle* h, int code, const char* msg) noexcept {
  if (h) {
    try {
      h->err = msg;
    } catch (...) {
    }
  }
  return code;
}

int fail(momenti_handle* h, int code, const std::string& msg) noexcept {
  if (h) {
    try {
      h->err = msg;
    } catch (...) {
    }
  }
  return code;
}

#define CK(call)                                                                       \
  do {                                                                                 \
    cudaError_t e_ = (call);                                                           \
    if (e_ != cudaSuccess)                                                             \
      return fail(h, MOMENTI_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
  } while (0)

// Device memory comes from one stream-ordered pool per device: a free is
// queued on the handle's stream (no device-wide synchronisation, so the
// handles of the batching form never stall one another) and freed blocks
// stay in the pool for the next allocation until momenti_destroy or the end
// of a batch trims it.
cudaMemPool_t lib_pool() {
  static std::mutex mu;
  static cudaMemPool_t pools[64] = {};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return nullptr;
  std::lock_guard<std::mutex> lk(mu);
  if (!pools[dev]) {
    cudaMemPoolProps pr{};
    pr.allocType = cudaMemAllocationTypePinned;
    pr.location.type = cudaMemLocationTypeDevice;
    pr.location.id = dev;
    cudaMemPool_t pool = nullptr;
    if (cudaMemPoolCreate(&pool, &pr) != cudaSuccess) return nullptr;
    uint64_t keep = ~uint64_t(0);
    cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
    pools[dev] = pool;
  }
  return pools[dev];
}

void trim_pool() {
  if (cudaMemPool_t pool = lib_pool()) cudaMemPoolTrimTo(pool, 0);
}

// Transient stream-ordered allocation from the library pool (memory the
// pool keeps is reused by the next call instead of being mapped again).
template <typename T>
cudaError_t pool_malloc(T** ptr, size_t bytes, cudaStream_t s) {
  cudaMemPool_t pool = lib_pool();
  if (!pool) return cudaErrorInitializationError;
  return cudaMallocFromPoolAsync(reinterpret_cast<void**>(ptr), std::max<size_t>(bytes, 16), pool, s);
}

template <typename T>
cudaError_t dalloc(momenti_handle* h, T** ptr, size_t count) {
  size_t bytes = std::max<size_t>(count * sizeof(T), 16);
  void* p = nullptr;
  cudaMemPool_t pool = lib_pool();
  if (!pool) return cudaErrorInitializationError;
  cudaError_t e = cudaMallocFromPoolAsync(&p, bytes, pool, h->stream);
  if (e != cudaSuccess) return e;
  h->bufs.push_back(DevBuf{p, bytes});
  h->device_bytes += bytes;
  *ptr = static_cast<T*>(p);
  return cudaSuccess;
}

// Releases the device buffers (queued on the handle's stream); the pinned
// host buffers survive unless `host` is set.
void free_all(momenti_handle* h, bool host = false) {
  for (auto& b : h->bufs) cudaFreeAsync(b.p, h->stream);
  h->bufs.clear();
  h->device_bytes = 0;
  if (host) {
    if (h->stream) cudaStreamSynchronize(h->stream);
    else cudaDeviceSynchronize();
    if (h->rec_host) cudaFreeHost(h->rec_host);
    if (h->cnt_host) cudaFreeHost(h->cnt_host);
    if (h->sort_cnt_host) cudaFreeHost(h->sort_cnt_host);
    h->sort_cnt_host = nullptr;
    h->rec_host = nullptr;
    h->cnt_host = nullptr;
    h->rec_host_cap = 0;
  }
  h->rec_dev = nullptr;
  h->draw_a = h->draw_u = nullptr;
  h->flags = nullptr;
  h->small = nullptr;
  h->jobs = nullptr;
  h->job_counts = nullptr;
  h->job_cap = 0;
  h->ix = Index{};
  h->sort = SortScratch{};
  h->cs = CollideScratch{};
  h->hs = HashSet{};
  h->ready = false;
}

// Work model of the traversal and of the exact path, in milliseconds on a
// GB300 (fitted to measured kernel times; only the ratio of the two
// predictions matters).  Per repetition of a level: pair tiles compared,
// sub-bucket pairs compared, events (each gets the segment-mean lower
// bound), full verifications, records handed to TOP on the host.
double predict_rep_ms(const Index& ix, uint64_t tiles, uint64_t sub_checks, uint64_t events,
                      uint64_t verified, uint64_t records) {
  const int G = (ix.D + 7) / 8;                    // byte-plane words per hash value
  const double tile_ns = G == 1 ? 3.0 : (G == 2 ? 4.1 : 5.3 * double(G));
  const double verify_ns = 2.0 * double(ix.w) * double(ix.Dp ? ix.Dp : ix.D) / 2400.0 + 0.5;
  return 1e-6 * (tile_ns * double(tiles) + 0.025 * double(sub_checks) + 0.8 * double(events) +
                 verify_ns * double(verified) + 100.0 * double(records));
}

// Recording sweeps the exact path is predicted to cost: one from a full
// TOP's k-th; without it, on a large series the slices start low and
// double (about two), otherwise the row-minima sweep, which computes every
// pair's distances in full (measured at about three recording sweeps at
// D = 8), comes first.
int exact_sweeps(const Index& ix, bool top_full) {
  if (top_full) return 1;
  const bool large = double(ix.M) * double(ix.M) * double(ix.D) > 4e11;
  return large ? 2 : 4;
}

double predict_exact_ms(const Index& ix, int passes) {
  double ps_pair;                                  // all-pairs kernel, per pair
  if (ix.xT && !ix.has_lo && ix.Dp == 4) ps_pair = 5.0;
  else if (ix.xT && !ix.has_lo && ix.Dp == 8) ps_pair = 7.5;
  else if (ix.xT && !ix.has_lo && ix.Dp == 16) ps_pair = 40.0;
  else if (ix.xW && rows2_usable(ix)) ps_pair = 1.5 * double(ix.DW);
  else if (ix.D <= 32) ps_pair = 8.0 * double(ix.D);
  else ps_pair = 31.0 * double(ix.D);
  const double pairs = 0.5 * double(ix.M) * double(ix.M);
  return double(passes) * (ps_pair * 1e-9 * pairs + 0.2) + 2.0;
}

// Bucket jobs of one chunk of repetitions (four lists by size, a quarter each)
uint64_t job_cap_for(int64_t M, int D) {
  uint64_t c = uint64_t(1) << 20;
  while (c < uint64_t(kChunkReps) * uint64_t(D) * uint64_t(M) && c < (uint64_t(1) << 25)) c <<= 1;
  return c;
}

int isqrt(int x) {
  int m = 0;
  while ((m + 1) * (m + 1) <= x) ++m;
  return m;
}

uint64_t next_pow2(uint64_t x) {
  uint64_t p = 1;
  while (p < x) p <<= 1;
  return p;
}

struct Timer {
  cudaEvent_t a = nullptr, b = nullptr;
  cudaStream_t s;
  explicit Timer(cudaStream_t st) : s(st) {
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    cudaEventRecord(a, s);
  }
  double stop() {
    cudaEventRecord(b, s);
    cudaEventSynchronize(b);
    float ms = 0;
    cudaEventElapsedTime(&ms, a, b);
    return ms;
  }
  ~Timer() {
    cudaEventDestroy(a);
    cudaEventDestroy(b);
  }
};

// Re-verifies in float64 every pool pair whose float32 dist_d is within
// tolerance of the k-th selected one, and selects the top-k again on the
// float64 distances.  fills out/n_out; returns the max relative float32
// error over the result.
int finalize(momenti_handle* h, int d, std::vector<PoolEntry> cand, momenti_motif* out,
             int32_t* n_out, double fail_bound, double* max_err) {
  const Index& ix = h->ix;
  const int k = h->p.k;
  std::sort(cand.begin(), cand.end(), pair_less);
  auto acc = greedy(cand, k, ix.excl);
  double kth = acc.empty() ? INFINITY : cand[acc.back()].dd;
  double lim = std::isfinite(kth) ? kth * (1.0 + 1e-4) + 1e-6 : INFINITY;
  std::vector<PoolEntry> near;
  for (auto& c : cand)
    if (c.dd <= lim) near.push_back(c);
  const int64_t m = int64_t(near.size());
  *max_err = 0.0;
  if (m > 0) {
    std::vector<uint64_t> pk(m);
    for (int64_t q = 0; q < m; ++q) pk[q] = (uint64_t(near[q].a) << 32) | near[q].b;
    uint64_t* dp = nullptr;
    double *dpd = nullptr, *ddd = nullptr;
    uint64_t* dmask = nullptr;
    CK(pool_malloc(&dp, m * 8, h->stream));
    CK(pool_malloc(&dpd, m * ix.D * 8, h->stream));
    CK(pool_malloc(&ddd, m * 8, h->stream));
    CK(pool_malloc(&dmask, m * 8, h->stream));
    CK(cudaMemcpyAsync(dp, pk.data(), m * 8, cudaMemcpyHostToDevice, h->stream));
    CK(launch_verify_pairs(ix, d, dp, m, 1, dpd, ddd, dmask, h->stream));
    std::vector<double> per(m * ix.D), dd(m);
    std::vector<uint64_t> mk(m);
    CK(cudaMemcpyAsync(per.data(), dpd, m * ix.D * 8, cudaMemcpyDeviceToHost, h->stream));
    CK(cudaMemcpyAsync(dd.data(), ddd, m * 8, cudaMemcpyDeviceToHost, h->stream));
    CK(cudaMemcpyAsync(mk.data(), dmask, m * 8, cudaMemcpyDeviceToHost, h->stream));
    CK(cudaFreeAsync(dp, h->stream));
    CK(cudaFreeAsync(dpd, h->stream));
    CK(cudaFreeAsync(ddd, h->stream));
    CK(cudaFreeAsync(dmask, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    for (int64_t q = 0; q < m; ++q) {
      double mx = 0;
      for (int f = 0; f < ix.D; ++f)
        if (mk[q] >> f & 1) mx = std::max(mx, per[q * ix.D + f]);
      near[q].dd = dd[q];
      near[q].dmax = mx;
      near[q].dims = mk[q];
    }
    std::sort(near.begin(), near.end(), pair_less);
    acc = greedy(near, k, ix.excl);
    cand = near;
  }
  int cnt = 0;
  for (size_t q : acc) {
    const PoolEntry& c = cand[q];
    out[cnt].a = c.a;
    out[cnt].b = c.b;
    out[cnt].dist_d = c.dd;
    out[cnt].dist_max = c.dmax;
    out[cnt].fail_bound = fail_bound;
    out[cnt].dims_mask = c.dims;
    ++cnt;
  }
  *n_out = cnt;
  return MOMENTI_OK;
}

// Exact all-pairs top-k (the final fallback of Algorithm 1).  tau0 <= 0: derive the
// first threshold from per-window nearest distances.
int exact_path(momenti_handle* h, int d, double tau0, momenti_motif* out, int32_t* n_out,
               double* max_err) {
  Index& ix = h->ix;
  const int k = h->p.k;
  // First threshold: TOP's k-th (tau0), else 1.2 x the 2k-th smallest row
  // minimum of spaced windows.  On a large series (M^2 D > 4e11) a loose
  // threshold costs a sweep in which most pairs pass the filters, and the
  // row-minima sweep evaluates every pair in full: there, when TOP holds
  // only background pairs (its k-th above a quarter of the largest possible
  // dist_d, 2 d sqrt(w)) or is not full, the slices start at 5% of that
  // largest value and double.  Any start gives the same exact result.
  const double dmax_all = 2.0 * double(d) * std::sqrt(double(ix.w));
  const double tau_low = 0.05 * dmax_all;
  const bool large = double(ix.M) * double(ix.M) * double(ix.D) > 4e11;
  double tau = tau0;
  if (large && (!(tau > 0) || tau > 0.25 * dmax_all)) tau = tau > 0 ? std::min(tau, tau_low) : tau_low;
  if (!(tau > 0)) {
    float* rowmin = nullptr;
    CK(pool_malloc(&rowmin, ix.M * 4, h->stream));
    CK(cudaMemsetAsync(rowmin, 0x7f, ix.M * 4, h->stream));
    const auto tr0 = std::chrono::steady_clock::now();
    CK(launch_allpairs_rowmin(ix, d, rowmin, h->stream));
    std::vector<float> rm(ix.M);
    CK(cudaMemcpyAsync(rm.data(), rowmin, ix.M * 4, cudaMemcpyDeviceToHost, h->stream));
    CK(cudaFreeAsync(rowmin, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    // 2k-th smallest nearest distance among windows spaced more than eps
    std::vector<std::pair<float, int64_t>> v;
    for (int64_t a = 0; a < ix.M; ++a)
      if (std::isfinite(rm[a])) v.push_back({rm[a], a});
    std::sort(v.begin(), v.end());
    std::vector<int64_t> picked;
    double val = 0;
    for (auto& pr : v) {
      bool ok = true;
      for (int64_t q : picked)
        if (std::llabs(q - pr.second) <= ix.excl) { ok = false; break; }
      if (!ok) continue;
      picked.push_back(pr.second);
      val = pr.first;
      if (int(picked.size()) >= 2 * k) break;
    }
    if (picked.empty()) {
      *n_out = 0;
      return MOMENTI_OK;
    }
    tau = std::max(val * 1.2, 1e-3);
    if (const char* t1 = std::getenv("MOMENTI_TRACE"); t1 && t1[0] == '1')
      std::fprintf(stderr, "momenti trace: exact row minima ms=%.1f\n",
                   std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - tr0).count());
  }
  if (const char* t0 = std::getenv("MOMENTI_TRACE"); t0 && t0[0] == '1')
    std::fprintf(stderr, "momenti trace: exact tau=%.5g (%s)\n", tau,
                 tau == tau0 ? "from TOP" : (tau == tau_low ? "low start" : "from row minima"));
  const auto te0 = std::chrono::steady_clock::now();
  // Pairs are taken in slices of their approximate dist_d (float32 Pearson
  // form, within 1% + 0.01 of the exact value): each all-pairs sweep records
  // the pairs with approximate distance in (lo, hi] and a histogram of them;
  // they are verified in ascending batches (float32, direct form) and added
  // to the candidates, and greedy runs after every batch.  Once every pair
  // with exact dist_d <= e is held (e = (edge - 0.01) / 1.01 for the upper
  // edge of what has been taken) and greedy's k-th is below e, the prefix is
  // exact.
  std::vector<PoolEntry> got;
  const char* tr = std::getenv("MOMENTI_TRACE");
  const bool trace = tr && tr[0] == '1';
  auto add_batch = [&](const uint64_t* dpairs, int64_t m) -> int {
    if (m <= 0) return MOMENTI_OK;
    double *dpd = nullptr, *ddd = nullptr;
    uint64_t* dmask = nullptr;
    CK(pool_malloc(&dpd, m * ix.D * 8, h->stream));
    CK(pool_malloc(&ddd, m * 8, h->stream));
    CK(pool_malloc(&dmask, m * 8, h->stream));
    CK(launch_verify_pairs(ix, d, dpairs, m, 0, dpd, ddd, dmask, h->stream));
    std::vector<uint64_t> pk(m), mk(m);
    std::vector<double> per(m * ix.D), dd(m);
    CK(cudaMemcpyAsync(pk.data(), dpairs, m * 8, cudaMemcpyDeviceToHost, h->stream));
    CK(cudaMemcpyAsync(per.data(), dpd, m * ix.D * 8, cudaMemcpyDeviceToHost, h->stream));
    CK(cudaMemcpyAsync(dd.data(), ddd, m * 8, cudaMemcpyDeviceToHost, h->stream));
    CK(cudaMemcpyAsync(mk.data(), dmask, m * 8, cudaMemcpyDeviceToHost, h->stream));
    CK(cudaFreeAsync(dpd, h->stream));
    CK(cudaFreeAsync(ddd, h->stream));
    CK(cudaFreeAsync(dmask, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    const size_t old_n = got.size();
    for (int64_t q = 0; q < m; ++q) {
      double mx = 0;
      for (int f = 0; f < ix.D; ++f)
        if (mk[q] >> f & 1) mx = std::max(mx, per[q * ix.D + f]);
      got.push_back(PoolEntry{dd[q], mx, uint32_t(pk[q] >> 32), uint32_t(pk[q]), mk[q]});
    }
    // got stays sorted: sort the batch, merge it in
    std::sort(got.begin() + old_n, got.end(), pair_less);
    std::inplace_merge(got.begin(), got.begin() + old_n, got.end(), pair_less);
    return MOMENTI_OK;
  };
  // greedy over everything taken; true when its k-th lies below e
  auto exact_below = [&](double e) -> bool {
    auto acc = greedy(got, k, ix.excl);
    return int(acc.size()) == k && got[acc.back()].dd * (1.0 + 1e-4) + 1e-6 <= e;
  };
  // no pair has an approximate distance above this
  const float all_edge = float(2.0 * std::sqrt(double(ix.w)) * d * 1.01 + 0.02);
  constexpr int64_t kBatch = int64_t(1) << 13;   // pairs verified per batch (smallest first)
  size_t free_b = 0, total_b = 0;
  CK(cudaMemGetInfo(&free_b, &total_b));
  const uint64_t cap_max = std::max<uint64_t>(uint64_t(1) << 22,
                                              std::min<uint64_t>(uint64_t(1) << 30, free_b / 4 / 12));
  uint64_t cap = std::min<uint64_t>(uint64_t(1) << 24, cap_max);
  float lo = -1.f;
  float hi = std::min(float(tau) * 1.01f + 1e-2f, all_edge);
  uint64_t* dout = nullptr;
  float* dval = nullptr;
  unsigned long long* dcnt = nullptr;
  uint32_t* dhist = nullptr;
  uint64_t* dsel = nullptr;
  auto release = [&]() {
    if (dout) cudaFreeAsync(dout, h->stream);
    if (dval) cudaFreeAsync(dval, h->stream);
    if (dsel) cudaFreeAsync(dsel, h->stream);
    dout = nullptr;
    dval = nullptr;
    dsel = nullptr;
  };
  CK(pool_malloc(&dcnt, 8, h->stream));
  CK(pool_malloc(&dhist, kApBins * 4, h->stream));
  std::vector<uint32_t> hist(kApBins);
  int rc = MOMENTI_ERR_OVERFLOW;
  for (int pass = 0; pass < 64; ++pass) {
    if (!dout) {
      CK(pool_malloc(&dout, cap * 8, h->stream));
      CK(pool_malloc(&dval, cap * 4, h->stream));
    }
    CK(cudaMemsetAsync(dcnt, 0, 8, h->stream));
    CK(cudaMemsetAsync(dhist, 0, kApBins * 4, h->stream));
    ApRec ar;
    ar.out = dout;
    ar.out_d = dval;
    ar.cap = cap;
    ar.count = dcnt;
    ar.hist = dhist;
    ar.lo = lo;
    ar.hscale = float(kApBins) / (hi - lo);
    const auto tp0 = std::chrono::steady_clock::now();
    if (h->batcher && sweep_batchable(ix))
      CK(h->batcher->sweep(ix, d, hi, ar, h->stream));
    else
      CK(launch_allpairs(ix, d, hi, ar, h->stream));
    unsigned long long cnt = 0;
    CK(cudaMemcpyAsync(&cnt, dcnt, 8, cudaMemcpyDeviceToHost, h->stream));
    CK(cudaMemcpyAsync(hist.data(), dhist, kApBins * 4, cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    if (trace)
      std::fprintf(stderr, "momenti trace: exact pass=%d lo=%.5g hi=%.5g pairs=%llu cap=%llu held=%zu ms=%.1f\n",
                   pass, double(lo), double(hi), cnt, (unsigned long long)cap, got.size(),
                   std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - tp0).count());
    const double width = double(hi - lo) / kApBins;
    if (cnt > cap) {
      // lower the upper edge to the largest bin edge whose pairs fit; grow
      // the buffer only when the first bin alone does not fit
      uint64_t run = 0;
      int bin = 0;
      for (; bin < kApBins; ++bin) {
        if (run + hist[bin] > cap) break;
        run += hist[bin];
      }
      if (bin > 0) {
        hi = float(double(lo) + width * bin);
      } else {
        release();
        if (uint64_t(hist[0]) > cap_max)
          return fail(h, MOMENTI_ERR_MEMORY, "exact path: one distance bin exceeds memory");
        cap = std::min<uint64_t>(cap_max, (uint64_t(cnt) + (uint64_t(1) << 20)) & ~((uint64_t(1) << 20) - 1));
      }
      continue;
    }
    // ascending batches of whole bins
    CK(pool_malloc(&dsel, std::max<uint64_t>(cnt, 1) * 8, h->stream));
    bool done = false;
    for (int b0 = 0; b0 < kApBins && !done;) {
      int b1 = b0;
      uint64_t run = 0;
      while (b1 < kApBins && (b1 == b0 || run + hist[b1] <= uint64_t(kBatch))) run += hist[b1++];
      const float slo = b0 == 0 ? lo : float(double(lo) + width * b0);
      const float shi = b1 == kApBins ? hi : float(double(lo) + width * b1);
      if (run > 0) {
        CK(cudaMemsetAsync(dcnt, 0, 8, h->stream));
        CK(launch_select_pairs(dout, dval, cnt, slo, shi, dsel, dcnt, h->stream));
        unsigned long long ns = 0;
        CK(cudaMemcpyAsync(&ns, dcnt, 8, cudaMemcpyDeviceToHost, h->stream));
        CK(cudaStreamSynchronize(h->stream));
        const int r = add_batch(dsel, int64_t(ns));
        if (r != MOMENTI_OK) return r;
      }
      done = exact_below((double(shi) - 1e-2) / 1.01);
      b0 = b1;
    }
    release();
    if (done || hi >= all_edge) {
      // done, or every pair is held: fewer than k non-trivial motifs exist
      rc = finalize(h, d, got, out, n_out, 0.0, max_err);
      break;
    }
    lo = hi;
    hi = std::min(2.f * hi + 1e-2f, all_edge);
  }
  cudaFreeAsync(dcnt, h->stream);
  cudaFreeAsync(dhist, h->stream);
  if (trace)
    std::fprintf(stderr, "momenti trace: exact done ms=%.1f\n",
                 std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - te0).count());
  if (rc == MOMENTI_ERR_OVERFLOW) return fail(h, rc, "exact path: threshold search did not converge");
  return rc;
}

}  // namespace

extern "C" {

int momenti_default_params(momenti_params* p) {
  if (!p) return MOMENTI_ERR_ARG;
  std::memset(p, 0, sizeof(*p));
  p->w = 100;
  p->d = 1;
  p->k = 1;
  p->delta = 0.01;
  p->mem_limit = 0;
  p->K = 8;
  p->L = 200;
  p->r = 0.0;
  p->excl = -1;
  p->seed = 0;
  p->precision = MOMENTI_PREC_F16X2;
  p->delta_mode = MOMENTI_DELTA_PER_MOTIF;
  return MOMENTI_OK;
}

static int create_impl(momenti_handle** out, const momenti_params* p) {
  if (!out || !p) return MOMENTI_ERR_ARG;
  *out = nullptr;
  if (p->w < 2 || p->d < 1 || p->k < 1 || !(p->delta > 0.0 && p->delta < 1.0) || p->K < 1 ||
      p->K > MOMENTI_MAX_K || p->L < 0 ||
      (p->precision != MOMENTI_PREC_FP32 && p->precision != MOMENTI_PREC_F16X2) ||
      (p->delta_mode != MOMENTI_DELTA_PER_MOTIF && p->delta_mode != MOMENTI_DELTA_ALL_K) ||
      ((p->flags & MOMENTI_FLAG_TENSORING) && (p->K % 2 != 0)))
    return MOMENTI_ERR_ARG;
  auto* h = new momenti_handle();
  h->p = *p;
  *out = h;
  return MOMENTI_OK;
}

void momenti_destroy(momenti_handle* h) {
  if (!h) return;
  free_all(h, true);
  if (h->own_stream) cudaStreamDestroy(h->own_stream);
  delete h;
  trim_pool();
}

const char* momenti_last_error(const momenti_handle* h) {
  if (!h) return "no handle";
  return h->err.c_str();
}

static int set_hash_params_impl(momenti_handle* h, int32_t D, int32_t L, int32_t K, int32_t w,
                            const float* a, const float* u) {
  if (!h) return MOMENTI_ERR_ARG;
  const bool tens = (h->p.flags & MOMENTI_FLAG_TENSORING) != 0;
  const int K_fn = tens ? h->p.K / 2 : h->p.K;      // values per hash function
  if (!a || !u || D < 1 || D > MOMENTI_MAX_D || L < 1 || K != K_fn || w != h->p.w ||
      (tens && L % 2 != 0))
    return fail(h, MOMENTI_ERR_ARG, "set_hash_params: bad sizes");
  const size_t na = size_t(D) * L * K * w, nu = size_t(D) * L * K;
  for (size_t q = 0; q < nu; ++q)
    if (!(u[q] >= 0.f && u[q] < 1.f)) return fail(h, MOMENTI_ERR_ARG, "set_hash_params: u outside [0,1)");
  h->user_a.assign(a, a + na);
  h->user_u.assign(u, u + nu);
  h->user_D = D;
  h->user_L = L;
  h->user_K = K;
  ++h->hp_gen;
  return MOMENTI_OK;
}

static int hash_all_impl(momenti_handle* h, const void* series, int32_t dtype, int64_t n, int32_t D,
                     int64_t ld, int32_t on_device, void* stream) {
  if (!h) return MOMENTI_ERR_ARG;
  const auto& p = h->p;
  const bool tens = (p.flags & MOMENTI_FLAG_TENSORING) != 0;
  if (!series || D < 1 || D > MOMENTI_MAX_D || p.d > D || n < p.w || ld < n ||
      (dtype != MOMENTI_F32 && dtype != MOMENTI_F64))
    return fail(h, MOMENTI_ERR_ARG, "hash_all: bad arguments");
  const int64_t M = n - p.w + 1;
  if (M >= kMaxWindows) return fail(h, MOMENTI_ERR_ARG, "hash_all: too many windows");
  if (!h->user_a.empty() && h->user_D != D)
    return fail(h, MOMENTI_ERR_ARG, "hash_all: D differs from set_hash_params");
  // a series of the same shape reuses every buffer of the previous index
  const bool reuse = h->ready && h->ix.n == n && h->ix.D == D &&
                     h->ix.has_lo == (dtype == MOMENTI_F64) && h->built_gen == h->hp_gen &&
                     std::memcmp(&h->built_p, &h->p, sizeof(momenti_params)) == 0;
  if (!reuse) free_all(h);
  h->ready = false;
  h->search.reset();                       // a search in progress ends with its index
  // buffers last used on another stream: let that work finish first
  if (h->stream != static_cast<cudaStream_t>(stream) && !h->bufs.empty())
    cudaStreamSynchronize(h->stream);
  h->stream = static_cast<cudaStream_t>(stream);
  cudaStream_t s = h->stream;
  Index& ix = h->ix;
  const int w = p.w, K = p.K;
  const size_t elem = dtype == MOMENTI_F64 ? 8 : 4;

  if (!reuse) {
    // ---- memory planner ----
    size_t free_b = 0, total_b = 0;
    CK(cudaMemGetInfo(&free_b, &total_b));
    const uint64_t limit = p.mem_limit ? p.mem_limit : uint64_t(0.8 * double(free_b));
    const int Wp = ((w + 63) / 64) * 64;
    const uint64_t fixed = uint64_t(D) * n * (dtype == MOMENTI_F64 ? 8 : 4)  // series hi/lo
                           + uint64_t(D) * n * elem                          // transient staging
                           + uint64_t(D) * M * (8 + 8 + 4 + 4 + 4)           // stats
                           + (D <= 16 ? uint64_t(16) * (3 * n + 4 * M) * 4 + M : 0)  // point-major copies
                           + (D > 16 ? uint64_t(64) * (n + M) * 4 + M : 0)   // point-major wide copy, column table
                           + (D <= 16 && p.d >= 2 ? job_cap_for(M, D) * sizeof(BucketJob) : 0)
                           + (uint64_t(64) << 20);                           // small scratch
    const uint64_t per_rep = uint64_t(M) * D * (8 + 4 + 1)                   // keys, order, lcp
                             + uint64_t(D) * kRepStride * Wp * (2 + 4)       // a16, a32
                             + uint64_t(D) * kRepStride * 4                  // boff
                             + uint64_t(D) * K * (w + 1) * 4                 // draws
                             + uint64_t(D) * M * kRepStride * 8 / 400;       // rehash flags (0.25%)
    const int L_cap = p.L > 0 ? p.L : 4096;
    int L_user = h->user_a.empty() ? L_cap : std::min(L_cap, h->user_L);
    if (tens && !h->user_a.empty()) L_user = std::min(L_cap, (h->user_L / 2) * (h->user_L / 2));
    // sort scratch: a batch of repetitions whose ping-pong buffers hold about 640 MB
    // (fewer, fuller launches; measured faster than batches that stay in L2)
    const uint64_t seg_bytes = uint64_t(M) * (8 + 8 + 4 + 4);
    int sort_reps = int(std::max<uint64_t>(1, (uint64_t(640) << 20) / (seg_bytes * D)));
    // traversal scratch
    const int64_t C = (M + 31) / 32;
    int chunk = std::min(kChunkReps, L_user);
    const uint64_t new_cap = uint64_t(1) << 21;
    const uint64_t hs_cap = std::min<uint64_t>(
        uint64_t(1) << 25, std::max<uint64_t>(uint64_t(1) << 20, next_pow2(uint64_t(M) * 64)));
    auto scratch_bytes = [&](int sreps, int creps) {
      return uint64_t(sort_scratch_bytes(M, sreps * D)) +
             uint64_t(creps) * D * (C + 1) * (4 + 4 + 8) + new_cap * 32 + hs_cap * 8 +
             (uint64_t(1) << 22) * sizeof(Event);
    };
    auto total_bytes = [&](int LL) {
      return fixed + scratch_bytes(std::min(sort_reps, LL), std::min(chunk, LL)) +
             uint64_t(LL) * per_rep;
    };
    if (total_bytes(1) > limit)
      return fail(h, MOMENTI_ERR_MEMORY, "hash_all: memory limit below one repetition");
    int L = L_user;
    if (total_bytes(L) > limit) {
      int lo = 1, hi = L;          // largest L that fits
      while (lo < hi) {
        int mid = (lo + hi + 1) / 2;
        if (total_bytes(mid) <= limit) lo = mid;
        else hi = mid - 1;
      }
      L = lo;
    }
    if (tens) {                            // tensoring: a square number of repetitions
      int m = 1;
      while ((m + 1) * (m + 1) <= L) ++m;
      L = m * m;
    }
    sort_reps = std::max(1, std::min(sort_reps, L));
    chunk = std::max(1, std::min(chunk, L));
    h->chunk_reps = chunk;
    h->sort_reps = sort_reps;

    ix.n = n;
    ix.M = M;
    ix.D = D;
    ix.w = w;
    ix.K = K;
    ix.L = L;
    ix.Wp = Wp;
    ix.excl = p.excl < 0 ? w / 2 : p.excl;
    ix.has_lo = dtype == MOMENTI_F64;
    // projections per dim: K per repetition, or K/2 per half function
    const int N = (tens ? 2 * isqrt(L) : L) * kRepStride;
    CK(dalloc(h, &ix.xs_hi, size_t(D) * n));
    if (ix.has_lo) CK(dalloc(h, &ix.xs_lo, size_t(D) * n));
    if (D > 16 && dtype == MOMENTI_F32) {       // the row-staged sweep of wide series
      ix.DW = D <= 32 ? 32 : 64;
      CK(dalloc(h, &ix.xW, size_t(ix.DW) * n));
      CK(dalloc(h, &ix.isW, size_t(ix.DW) * M));
      CK(dalloc(h, &ix.cflag, size_t(M)));
    }
    if (D <= 16) {
      ix.Dp = D <= 4 ? 4 : (D <= 8 ? 8 : 16);
      CK(dalloc(h, &ix.xT, size_t(ix.Dp) * n));
      CK(dalloc(h, &ix.stT, size_t(3) * ix.Dp * M));
      if (!ix.has_lo) {
        CK(dalloc(h, &ix.isT, size_t(ix.Dp) * M));
        CK(dalloc(h, &ix.cflag, size_t(M)));
      }
      if (ix.has_lo) CK(dalloc(h, &ix.xlT, size_t(ix.Dp) * n));
      if (w >= 32) {
        CK(dalloc(h, &ix.smT, size_t(ix.Dp) * n));
        // padding dims stay zero
        CK(cudaMemsetAsync(ix.smT, 0, size_t(ix.Dp) * n * 4, static_cast<cudaStream_t>(stream)));
      }
    }
    CK(dalloc(h, &ix.mu, size_t(D) * M));
    CK(dalloc(h, &ix.sig, size_t(D) * M));
    CK(dalloc(h, &ix.mu_hi, size_t(D) * M));
    CK(dalloc(h, &ix.mu_lo, size_t(D) * M));
    CK(dalloc(h, &ix.inv_sig, size_t(D) * M));
    CK(dalloc(h, &ix.a16, size_t(D) * N * Wp));
    CK(dalloc(h, &ix.a32, size_t(D) * N * Wp));
    CK(dalloc(h, &ix.boff, size_t(D) * N));
    CK(dalloc(h, &ix.keys, size_t(L) * M * D));
    CK(dalloc(h, &ix.order, size_t(L) * M * D));
    CK(dalloc(h, &ix.lcp, size_t(L) * M * D));
    h->draw_a = nullptr;
    h->draw_u = nullptr;
    const int n_fn = tens ? 2 * isqrt(L) : L;          // hash functions per dim
    const int K_fn = tens ? K / 2 : K;                 // values per hash function
    const size_t na = h->user_a.empty() ? size_t(D) * n_fn * K_fn * w : h->user_a.size();
    const size_t nu = h->user_a.empty() ? size_t(D) * n_fn * K_fn : h->user_u.size();
    CK(dalloc(h, &h->draw_a, na));
    CK(dalloc(h, &h->draw_u, nu));
    // near-boundary values of the tensor-core form (about 0.1% of them; room
    // for 0.25%, beyond which the projections are redone in float32)
    h->flag_cap = uint32_t(std::min<uint64_t>(uint64_t(1) << 28,
                                              std::max<uint64_t>(uint64_t(1) << 16, uint64_t(D) * M * N / 400)));
    CK(dalloc(h, &h->flags, size_t(h->flag_cap)));
    CK(dalloc(h, &h->small, 16));
    // index sort scratch
    unsigned char* sort_region = nullptr;
    CK(dalloc(h, &sort_region, sort_scratch_bytes(M, sort_reps * D)));
    h->sort = sort_scratch_carve(sort_region, M, sort_reps * D);
    // traversal scratch
    CollideScratch& cs = h->cs;
    cs.seg_cap = int64_t(chunk) * D;
    cs.chunk_cap = C;
    const int64_t E = cs.seg_cap * C;
    CK(dalloc(h, &cs.cagg, size_t(E)));
    CK(dalloc(h, &cs.cbs, size_t(E)));
    CK(dalloc(h, &cs.ntile, size_t(E + 1)));
    CK(dalloc(h, &cs.scan_tmp, size_t(E / 1024 + 2)));
    CK(dalloc(h, &cs.counters, 8));
    h->rec_cap = new_cap;
    CK(dalloc(h, &h->rec_dev, size_t(new_cap)));
    HashSet& hs = h->hs;
    hs.cap = hs_cap;
    CK(dalloc(h, &hs.keys, size_t(hs_cap)));
    if (D <= 16 && p.d >= 2) {
      h->job_cap = job_cap_for(M, D);
      CK(dalloc(h, &h->jobs, size_t(h->job_cap)));
      CK(dalloc(h, &h->job_counts, 8));
    }
    cs.ev_cap = uint64_t(1) << 22;
    h->ev_budget = std::max<uint64_t>(uint64_t(1) << 28, limit / 8);
    CK(dalloc(h, &cs.events, size_t(cs.ev_cap)));
    if (h->rec_host_cap < new_cap) {
      if (h->rec_host) {
        cudaStreamSynchronize(s);
        cudaFreeHost(h->rec_host);
        h->rec_host = nullptr;
      }
      h->rec_host_cap = 0;
      CK(cudaMallocHost(&h->rec_host, new_cap * sizeof(PairRec)));
      h->rec_host_cap = new_cap;
    }
    if (!h->cnt_host) CK(cudaMallocHost(&h->cnt_host, 8 * sizeof(unsigned long long)));
    if (!h->sort_cnt_host) CK(cudaMallocHost(&h->sort_cnt_host, 64 * sizeof(uint32_t)));
    h->sort.host_cnt = h->sort_cnt_host;
    h->built_gen = h->hp_gen;
    h->built_p = h->p;
  }
  const int L = ix.L;
  // the functions that are projected: the repetitions themselves, or under
  // tensoring the 2m half functions of K/2 values, whose keys are then
  // interleaved into the m^2 repetitions' keys
  const int m_t = tens ? isqrt(L) : 0;
  Index hx = ix;
  uint64_t* half = nullptr;
  if (tens) {
    hx.L = 2 * m_t;
    hx.K = K / 2;
    CK(pool_malloc(&half, size_t(hx.L) * M * D * 8, s));
    hx.keys = half;
  }

  Timer t_all(s);
  // ---- series: device split into float32 hi (+ lo for float64 input) ----
  const void* src = series;
  void* staging = nullptr;
  if (!on_device) {
    CK(pool_malloc(&staging, size_t(D) * n * elem, s));
    CK(cudaMemcpy2DAsync(staging, n * elem, series, ld * elem, n * elem, D, cudaMemcpyHostToDevice, s));
    src = staging;
    ld = n;
  }
  CK(launch_split_series(src, dtype, n, D, ld, ix.xs_hi, ix.xs_lo, s));
  CK(launch_point_major(ix, s));
  if (staging) CK(cudaFreeAsync(staging, s));
  CK(launch_window_stats(ix, s));
  CK(launch_stats_point_major(ix, s));
  CK(launch_col_prep(ix, s));

  // ---- hash functions ----
  int L_src = hx.L;
  if (!h->user_a.empty()) {
    L_src = h->user_L;
    CK(cudaMemcpyAsync(h->draw_a, h->user_a.data(), h->user_a.size() * 4, cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(h->draw_u, h->user_u.data(), h->user_u.size() * 4, cudaMemcpyHostToDevice, s));
  } else {
    CK(launch_draw_hash(p.seed, D, hx.L, hx.K, w, h->draw_a, h->draw_u, s));
  }
  CK(launch_layout_hash(hx, h->draw_a, L_src, s));

  // ---- r: fixed, or Section 6.1's heuristic ----
  if (p.r > 0) {
    ix.r = p.r;
  } else {
    float* mm = reinterpret_cast<float*>(h->small);
    const float init[2] = {INFINITY, -INFINITY};
    CK(cudaMemcpyAsync(mm, init, 8, cudaMemcpyHostToDevice, s));
    const int S = int(std::min<int64_t>(M, 4096));
    CK(launch_r_sample(hx, S, mm, s));
    float res[2];
    CK(cudaMemcpyAsync(res, mm, 8, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    double rr = (double(res[1]) - double(res[0])) / 256.0;
    ix.r = (rr > 0 && std::isfinite(rr)) ? rr : 1.0;
  }
  ix.inv_r = float(1.0 / ix.r);
  hx.r = ix.r;
  hx.inv_r = ix.inv_r;
  CK(launch_layout_boff(hx, h->draw_u, L_src, s));

  // ---- projections and hashes of all repetitions ----
  h->used_tc = false;
  h->n_flagged = 0;
  if (p.precision == MOMENTI_PREC_F16X2 && tc_supported() &&
      proj_hash_tc_smem(ix.Wp, ix.has_lo) <= size_t(227) * 1024) {
    uint32_t* fcount = reinterpret_cast<uint32_t*>(h->small) + 2;
    int* err = reinterpret_cast<int*>(h->small) + 3;
    CK(cudaMemsetAsync(fcount, 0, 8, s));
    CK(launch_proj_hash_tc(hx, 0, hx.L, h->flags, h->flag_cap, fcount, err, s));
    CK(launch_rehash_fp32(hx, h->flags, fcount, h->flag_cap, s));
    uint32_t hc[2] = {0, 0};
    CK(cudaMemcpyAsync(hc, fcount, 8, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    if (hc[1]) return fail(h, MOMENTI_ERR_TIMEOUT, "hash_all: tensor-core projection wait timed out");
    h->n_flagged = hc[0];
    if (hc[0] > h->flag_cap) CK(launch_proj_hash_fp32(hx, 0, hx.L, s));   // flag list overflowed
    else h->used_tc = true;
  } else {
    CK(launch_proj_hash_fp32(hx, 0, hx.L, s));
  }
  if (tens) {
    CK(launch_tensor_keys(ix, half, m_t, 0, L, s));
    CK(cudaFreeAsync(half, s));
  }

  // ---- index: sort every (j, f) ----
  Timer t_sort(s);
  for (int j0 = 0; j0 < L; j0 += h->sort_reps)
    CK(launch_sort_reps(ix, j0, std::min(L, j0 + h->sort_reps), h->sort, s));
  h->t_sort_ms = t_sort.stop();
  h->t_hash_ms = t_all.stop();
  CK(cudaGetLastError());
  h->ready = true;
  return MOMENTI_OK;
}

// Algorithm 1 for the dimensionalities d_low..d_high (Section 6.3; one d
// is Algorithm 1 as printed), as a resumable search.  One TOP per d;
// collisions use W >= d_cur, the smallest d not yet confirmed; every
// verified pair is offered to the TOP of every unconfirmed d (its
// per-dimension distances give dist_d for all d); after each repetition
// every unconfirmed d whose TOP passes STOP with its own d is confirmed at
// that (i, j).  A confirmation that raises d_cur in the middle of a chunk
// of repetitions discards the rest of the chunk, clears the device set of
// verified pairs (its entries were found under the old condition) and runs
// the rest again under the new one, so the device follows the printed loop
// repetition by repetition.  Each d left unconfirmed gets the exact top-k.
static int search_begin_impl(momenti_handle* h, int d_low, int d_high) {
  if (!h) return MOMENTI_ERR_ARG;
  if (!h->ready) return fail(h, MOMENTI_ERR_STATE, "search before hash_all");
  const Index& ix = h->ix;
  if (d_low < 1 || d_high < d_low || d_high > ix.D)
    return fail(h, MOMENTI_ERR_ARG, "search: need 1 <= d_low <= d_high <= D");
  auto ss = std::make_unique<SearchState>();
  ss->d_low = d_low;
  ss->d_high = d_high;
  ss->ds.resize(size_t(d_high - d_low + 1));
  for (int q = 0; q <= d_high - d_low; ++q) {
    ss->ds[size_t(q)].d = d_low + q;
    ss->ds[size_t(q)].pool.k = h->p.k;
    ss->ds[size_t(q)].pool.eps = ix.excl;
  }
  ss->i = ix.K;
  ss->j0 = 0;
  ss->d_cur = d_low;
  ss->st.K = ix.K;
  ss->st.L = ix.L;
  ss->st.r = ix.r;
  ss->st.n_windows = ix.M;
  CK(launch_hashset_clear(h->hs, h->stream));
  h->set_fill = 0;
  h->search = std::move(ss);
  return MOMENTI_OK;
}

// Runs chunks of repetitions until max_reps repetitions have been processed
// (at least one chunk) or the traversal has ended.
static int search_step_impl(momenti_handle* h, int64_t max_reps, int32_t* ended) {
  if (!h) return MOMENTI_ERR_ARG;
  if (!h->search) return fail(h, MOMENTI_ERR_STATE, "search_step without search_begin");
  SearchState& S = *h->search;
  Index& ix = h->ix;
  const auto& p = h->p;
  cudaStream_t s = h->stream;
  const int K = ix.K, L = ix.L, k = p.k;
  const int nd = S.d_high - S.d_low + 1;
  const bool tens = (p.flags & MOMENTI_FLAG_TENSORING) != 0;
  const double delta = p.delta_mode == MOMENTI_DELTA_ALL_K ? p.delta / k : p.delta;
  momenti_stats& st = S.st;
  std::vector<DState>& ds = S.ds;
  auto open_min = [&]() {
    for (auto& x : ds)
      if (!x.done) return x.d;
    return 0;
  };
  std::vector<std::vector<PairRec>> by_rep(h->chunk_reps);
  std::vector<PairRec> recd;                 // one record per dimensionality (several d)
  std::vector<double> per_dim, srt;
  unsigned long long* cnt = h->cnt_host;
  // MOMENTI_TRACE=1 prints one line per chunk (level, repetitions, work counts, TOP state)
  const char* tr = std::getenv("MOMENTI_TRACE");
  const bool trace = tr && tr[0] == '1';
  // cost switch: each level opens with a one-repetition probe
  const bool cost_switch = !(p.flags & MOMENTI_FLAG_NO_COST_SWITCH) && L > 1;
  Timer t_trav(s);
  int64_t reps_done = 0;
  while (!S.ended && (reps_done == 0 || reps_done < max_reps)) {
    if (S.j0 >= L) {                         // the level is complete
      S.j0 = 0;
      if (--S.i < 1) {
        S.ended = true;
        break;
      }
    }
    const int i = S.i, j0 = S.j0;
    const bool probe = cost_switch && j0 == 0;
    int j1 = probe ? 1 : std::min(L, j0 + h->chunk_reps);
    if (max_reps > 0 && j1 - j0 > max_reps - reps_done)          // the caller's step size
      j1 = j0 + int(std::max<int64_t>(1, max_reps - reps_done));
    const int d = S.d_cur;
    // device threshold: a pair is kept if it may enter the TOP of some
    // unconfirmed d (dist_d >= dist_{d_cur})
    float tau = 0.f;
    for (auto& x : ds)
      if (!x.done) tau = std::max(tau, x.tau);
    const auto tc0 = std::chrono::steady_clock::now();
    bool used_sub = false;
    unsigned long long tiles = 0;
    // collision counting (prefix length 1: buckets split by a second
    // dimension when every bucket fits a CTA); grow the event list, or
    // halve the chunk beyond the event budget
    for (;;) {
      bool sub = false;
      unsigned long long jc[5] = {0, 0, 0, 0, 0};
      if (i <= 3 && d >= 2 && ix.D <= 16 && h->jobs && !(p.flags & MOMENTI_FLAG_TILES_ONLY)) {
        CK(cudaMemsetAsync(h->job_counts, 0, 5 * sizeof(unsigned long long), s));
        CK(launch_bucket_jobs(ix, i, j0, j1, d, h->jobs, h->job_cap, h->job_counts, s));
        CK(cudaMemcpyAsync(jc, h->job_counts, sizeof(jc), cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        const uint64_t qcap = h->job_cap / 4;
        sub = jc[0] <= qcap && jc[2] <= qcap && jc[3] <= qcap && jc[4] <= qcap &&
              jc[1] <= uint64_t(subbucket_cap(ix.D, i));
      }
      CK(cudaMemsetAsync(h->cs.counters, 0, 8 * sizeof(unsigned long long), s));
      used_sub = sub;
      if (sub) {
        CK(launch_subbucket(ix, i, j0, j1, d, h->hs, h->cs, h->jobs, h->job_cap, h->job_counts,
                            int(jc[1]), s));
      } else {
        CK(launch_collide(ix, i, j0, j1, d, h->hs, h->cs, 0, nullptr, 0, s));
        const int64_t E = int64_t(j1 - j0) * ix.D * ((ix.M + 31) / 32);
        CK(cudaMemcpyAsync(&cnt[5], h->cs.ntile + E, sizeof(unsigned long long), cudaMemcpyDeviceToHost, s));
      }
      CK(cudaMemcpyAsync(cnt, h->cs.counters, 5 * sizeof(unsigned long long), cudaMemcpyDeviceToHost, s));
      if (sub) CK(cudaMemcpyAsync(&cnt[5], h->cs.counters + 5, sizeof(unsigned long long), cudaMemcpyDeviceToHost, s));
      CK(cudaStreamSynchronize(s));
      tiles = cnt[5];
      if (cnt[0] <= h->cs.ev_cap) break;
      const uint64_t cap = next_pow2(cnt[0]);
      if (cap * sizeof(Event) > h->ev_budget && j1 - j0 > 1) {
        j1 = j0 + (j1 - j0) / 2;
        continue;
      }
      Event* ev = nullptr;
      CK(dalloc(h, &ev, size_t(cap)));
      h->cs.events = ev;
      h->cs.ev_cap = cap;
    }
    st.n_candidates += int64_t(cnt[0]);
    st.n_verified += int64_t(cnt[0]);
    const uint64_t checks = used_sub ? tiles : tiles * 1024;
    st.n_pair_checks += int64_t(checks);
    const uint64_t n_events = cnt[0];
    uint64_t nrec = 0;
    if (cnt[0]) {
      for (;;) {
        CK(launch_verify_events(ix, d, h->hs, h->cs, tau, h->rec_dev, h->rec_cap, s));
        CK(cudaMemcpyAsync(cnt, h->cs.counters, 8 * sizeof(unsigned long long), cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        if (cnt[1] <= h->rec_cap) break;
        // grow the record buffers and verify the chunk's events again
        const uint64_t cap = next_pow2(cnt[1]);
        PairRec* rec = nullptr;
        CK(dalloc(h, &rec, size_t(cap)));
        if (h->rec_host_cap < cap) {
          PairRec* rh = nullptr;
          CK(cudaMallocHost(&rh, cap * sizeof(PairRec)));
          cudaFreeHost(h->rec_host);
          h->rec_host = rh;
          h->rec_host_cap = cap;
        }
        h->rec_dev = rec;
        h->rec_cap = cap;
        CK(cudaMemsetAsync(h->cs.counters + 1, 0, 7 * sizeof(unsigned long long), s));
      }
      nrec = cnt[1];
      h->set_fill += cnt[2];
      if (nrec) {
        CK(cudaMemcpyAsync(h->rec_host, h->rec_dev, nrec * sizeof(PairRec), cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
      }
    }
    // several dimensionalities: the per-dimension distances of every
    // record (the float32 form of the verification), and from them
    // dist_d, dist_d^max and dims_d for each d of the range
    if (nd > 1 && nrec) {
      std::vector<uint64_t> pk(nrec);
      for (uint64_t q = 0; q < nrec; ++q)
        pk[q] = (uint64_t(h->rec_host[q].a) << 32) | h->rec_host[q].b;
      uint64_t* dp = nullptr;
      double* dpd = nullptr;
      CK(pool_malloc(&dp, nrec * 8, s));
      CK(pool_malloc(&dpd, nrec * ix.D * 8, s));
      CK(cudaMemcpyAsync(dp, pk.data(), nrec * 8, cudaMemcpyHostToDevice, s));
      CK(launch_verify_pairs(ix, d, dp, int64_t(nrec), 0, dpd, nullptr, nullptr, s));
      per_dim.resize(nrec * ix.D);
      CK(cudaMemcpyAsync(per_dim.data(), dpd, nrec * ix.D * 8, cudaMemcpyDeviceToHost, s));
      CK(cudaFreeAsync(dp, s));
      CK(cudaFreeAsync(dpd, s));
      CK(cudaStreamSynchronize(s));
    }
    if (h->set_fill * 2 > h->hs.cap) {
      CK(launch_hashset_clear(h->hs, s));
      h->set_fill = 0;
    }
    ++st.n_chunks;
    const auto th0 = std::chrono::steady_clock::now();
    st.n_lb_pruned += int64_t(cnt[3]);
    for (auto& v : by_rep) v.clear();
    for (uint64_t q = 0; q < nrec; ++q) {
      int jj = h->rec_host[q].j - j0;
      if (jj < 0 || jj >= j1 - j0) return fail(h, MOMENTI_ERR_CUDA, "topk: bad repetition tag");
      PairRec rr = h->rec_host[q];
      rr.pad = uint32_t(q);                // row of the record's per-dimension distances
      by_rep[jj].push_back(rr);
    }
    for (int j = j0; j < j1; ++j) {
      auto& v = by_rep[j - j0];
      for (auto& x : ds) {
        if (x.done || v.empty()) continue;
        if (nd == 1) {
          x.pool.add(v.data(), v.size());
          continue;
        }
        // this d's distances: the sum of the d smallest per-dimension ones
        recd.assign(v.begin(), v.end());
        std::vector<int> ord(static_cast<size_t>(ix.D));
        for (auto& rc : recd) {
          const double* pd = per_dim.data() + size_t(rc.pad) * ix.D;
          srt.assign(pd, pd + ix.D);
          for (int f = 0; f < ix.D; ++f) ord[size_t(f)] = f;
          std::stable_sort(ord.begin(), ord.end(),
                           [&](int u, int w2) { return srt[size_t(u)] < srt[size_t(w2)]; });
          double sum = 0.0, mx = 0.0;
          uint64_t mask = 0;
          for (int q = 0; q < x.d; ++q) {
            const double val = srt[size_t(ord[size_t(q)])];
            sum += val;
            mx = std::max(mx, val);
            mask |= uint64_t(1) << ord[size_t(q)];
          }
          rc.dist_d = float(sum);
          rc.dist_max = float(mx);
          rc.dims = mask;
        }
        x.pool.add(recd.data(), recd.size());
      }
      S.last_i = i;
      S.last_j = j + 1;
      ++reps_done;
      bool confirmed = false;
      for (auto& x : ds) {
        if (x.done || !x.pool.valid()) continue;
        const double pr = std::pow(collision_probability(x.pool.top.back().dmax, ix.r), x.d);
        const double fbx = tens ? momenti_tensoring_failure_bound(pr, i, j + 1, K, L)
                                : failure_bound(x.pool.top.back().dmax, i, j + 1, K, L, x.d, ix.r);
        if (fbx <= delta) {
          x.done = true;
          x.stop_i = i;
          x.stop_j = j + 1;
          x.fb = fbx;
          confirmed = true;
        }
      }
      if (confirmed) {
        const int nc = open_min();
        if (nc != S.d_cur) {
          S.d_cur = nc;
          if (!nc) S.ended = true;
          if (nc && j + 1 < j1) {
            // the rest of the chunk ran under the old condition: again
            CK(launch_hashset_clear(h->hs, s));
            h->set_fill = 0;
            j1 = j + 1;
          }
          break;
        }
      }
    }
    S.j0 = j1;
    const auto tc1 = std::chrono::steady_clock::now();
    st.t_host_ms += std::chrono::duration<double, std::milli>(tc1 - th0).count();
    if (trace)
      std::fprintf(stderr,
                   "momenti trace: i=%d j=[%d,%d) d=%d sub=%d events=%llu tiles=%llu lb_pruned=%llu "
                   "records=%llu top=%d kth=%.5g ms=%.3f\n",
                   i, j0, j1, d, int(used_sub), cnt[0], tiles, cnt[3], (unsigned long long)nrec,
                   int(ds[0].pool.top.size()), ds[0].pool.top.empty() ? -1.0 : ds[0].pool.kth(),
                   std::chrono::duration<double, std::milli>(tc1 - tc0).count());
    for (auto& x : ds) {
      if (x.done || int(x.pool.top.size()) != k) continue;
      const float t2 = float(1.1 * x.pool.kth() + 1e-6);
      if (t2 < x.tau) x.tau = t2;
      x.pool.tau_trunc = std::min(x.pool.tau_trunc, double(x.tau));
    }
    if (probe && !S.ended) {
      // the rest of this level, and the lower levels, against the exact
      // path of every open d.  Shorter prefixes collide more, so each lower
      // level costs at least as much as this one; it is taken to grow by
      // the factor g this level's probe grew by over the previous level's,
      // kept within [1, 4]
      const uint64_t verified = n_events - std::min<uint64_t>(n_events, cnt[3]);
      const double rep = predict_rep_ms(ix, used_sub ? 0 : tiles, used_sub ? tiles : 0, n_events,
                                        verified, nrec);
      const double g = S.prev_rep_ms > 0.0 ? std::min(4.0, std::max(1.0, rep / S.prev_rep_ms)) : 1.0;
      S.prev_rep_ms = rep;
      double lower = 0.0, gl = 1.0;
      for (int l = i - 1; l >= 1; --l) {
        gl *= g;
        lower += gl;
      }
      const double rest = double(L - 1) * rep + lower * double(L) * rep;
      double exact = 0.0;
      for (auto& x : ds)
        if (!x.done) exact += predict_exact_ms(ix, exact_sweeps(ix, int(x.pool.top.size()) == k));
      if (rest > exact) {
        S.switch_level = i;
        S.ended = true;
        st.predicted_rest_ms = rest;
        st.predicted_exact_ms = exact;
      }
    }
  }
  st.t_traverse_ms += t_trav.stop();
  if (ended) *ended = S.ended ? 1 : 0;
  return MOMENTI_OK;
}

// TOP of every d now (the anytime property: each candidate comes with the
// miss-probability bound of its own dist_d^max after the repetitions done
// so far).  Distances are those of the traversal (float32 form).
static int search_current_impl(momenti_handle* h, momenti_motif* out, int32_t* n_out,
                               int32_t* cursor) {
  if (!h) return MOMENTI_ERR_ARG;
  if (!h->search) return fail(h, MOMENTI_ERR_STATE, "search_current without search_begin");
  if (!out || !n_out) return fail(h, MOMENTI_ERR_ARG, "search_current: NULL output");
  const SearchState& S = *h->search;
  const Index& ix = h->ix;
  const int k = h->p.k;
  const bool tens = (h->p.flags & MOMENTI_FLAG_TENSORING) != 0;
  for (size_t q = 0; q < S.ds.size(); ++q) {
    const DState& x = S.ds[q];
    int c = 0;
    for (const PoolEntry& e : x.pool.top) {
      momenti_motif& m = out[q * size_t(k) + size_t(c)];
      m.a = e.a;
      m.b = e.b;
      m.dist_d = e.dd;
      m.dist_max = e.dmax;
      m.dims_mask = e.dims;
      double fb = 1.0;
      if (x.done) {
        fb = x.fb;
      } else if (S.last_j > 0) {
        const double pr = std::pow(collision_probability(e.dmax, ix.r), x.d);
        fb = tens ? momenti_tensoring_failure_bound(pr, S.last_i, S.last_j, ix.K, ix.L)
                  : failure_bound(e.dmax, S.last_i, S.last_j, ix.K, ix.L, x.d, ix.r);
      }
      m.fail_bound = fb;
      if (++c == k) break;
    }
    n_out[q] = c;
  }
  if (cursor) {
    cursor[0] = S.last_i;
    cursor[1] = S.last_j;
    cursor[2] = S.ended ? 1 : 0;
  }
  return MOMENTI_OK;
}

// Completes the search: the rest of the traversal, then each d's result
// (float64 re-verified; the exact top-k for a d that STOP did not confirm).
// out holds k motifs per d, n_out and stops (i, j per d, 0 0 for the exact
// path) one entry per d.  The search ends with this call.
static int search_finish_impl(momenti_handle* h, momenti_motif* out, int32_t* n_out,
                              int32_t* stops, momenti_stats* stats) {
  if (!h) return MOMENTI_ERR_ARG;
  if (!h->search) return fail(h, MOMENTI_ERR_STATE, "search_finish without search_begin");
  if (!out || !n_out) return fail(h, MOMENTI_ERR_ARG, "topk: NULL output");
  while (!h->search->ended) {
    int r = search_step_impl(h, int64_t(1) << 40, nullptr);
    if (r != MOMENTI_OK) return r;
  }
  SearchState& S = *h->search;
  cudaStream_t s = h->stream;
  const int k = h->p.k;
  momenti_stats& st = S.st;
  st.switch_level = S.switch_level;
  double max_err = 0;
  Timer t_fb(s);
  bool any_exact = false;
  for (size_t q = 0; q < S.ds.size(); ++q) {
    DState& x = S.ds[q];
    momenti_motif* o = out + q * size_t(k);
    int32_t* no = n_out + q;
    st.n_pool += int64_t(x.pool.items.size());
    x.pool.sort_all();
    double err = 0;
    int rc;
    if (x.done) {
      // every pool pair at or below the k-th, for the float64 re-check
      std::vector<PoolEntry> cand;
      const double lim = x.pool.kth() * (1.0 + 1e-3) + 1e-5;
      for (auto& c : x.pool.items)
        if (c.dd <= lim) cand.push_back(c);
      rc = finalize(h, x.d, cand, o, no, x.fb, &err);
    } else {
      any_exact = true;
      double tau0 = (int(x.pool.top.size()) == k) ? x.pool.kth() * 1.05 + 1e-6 : 0.0;
      rc = exact_path(h, x.d, tau0, o, no, &err);
    }
    if (rc != MOMENTI_OK) return rc;
    // float32 traversal distances vs the float64 result
    for (int t = 0; t < *no; ++t) {
      uint64_t key = (uint64_t(o[t].a) << 32) | uint64_t(o[t].b);
      for (auto& c : x.pool.items)
        if (((uint64_t(c.a) << 32) | c.b) == key && o[t].dist_d > 0)
          err = std::max(err, std::fabs(c.dd - o[t].dist_d) / o[t].dist_d);
    }
    max_err = std::max(max_err, err);
    if (stops) {
      stops[2 * q] = x.stop_i;
      stops[2 * q + 1] = x.stop_j;
    }
  }
  st.t_fallback_ms = any_exact ? t_fb.stop() : 0.0;
  st.fallback = any_exact ? 1 : 0;
  st.stop_i = S.ds[0].stop_i;
  st.stop_j = S.ds[0].stop_j;
  st.max_rel_err_fp32 = max_err;
  st.t_hash_ms = h->t_hash_ms;
  st.t_sort_ms = h->t_sort_ms;
  st.device_bytes = h->device_bytes;
  st.precision_used = h->used_tc ? MOMENTI_PREC_F16X2 : MOMENTI_PREC_FP32;
  st.n_rehashed = h->n_flagged;
  if (stats) *stats = st;
  h->search.reset();
  return MOMENTI_OK;
}

static int topk_core(momenti_handle* h, int d_low, int d_high, momenti_motif* out, int32_t* n_out,
                     int32_t* stops, momenti_stats* stats) {
  if (!h) return MOMENTI_ERR_ARG;
  if (!out || !n_out) return fail(h, MOMENTI_ERR_ARG, "topk: NULL output");
  if (!h->ready) return fail(h, MOMENTI_ERR_STATE, "topk before hash_all");
  int r = search_begin_impl(h, d_low, d_high);
  if (r != MOMENTI_OK) return r;
  r = search_finish_impl(h, out, n_out, stops, stats);
  h->search.reset();
  return r;
}

static int topk_impl(momenti_handle* h, momenti_motif* out, int32_t* n_out, momenti_stats* stats) {
  if (!h) return MOMENTI_ERR_ARG;
  return topk_core(h, h->p.d, h->p.d, out, n_out, nullptr, stats);
}

static int topk_exact_impl(momenti_handle* h, momenti_motif* out, int32_t* n_out) {
  if (!h) return MOMENTI_ERR_ARG;
  if (!out || !n_out) return fail(h, MOMENTI_ERR_ARG, "topk_exact: NULL output");
  if (!h->ready) return fail(h, MOMENTI_ERR_STATE, "topk_exact before hash_all");
  double err = 0;
  return exact_path(h, h->p.d, 0.0, out, n_out, &err);
}

static int topk_batch_impl(int32_t B, const momenti_params* params, const void* const* series,
                       const int32_t* dtype, const int64_t* n, const int32_t* D, int32_t on_device,
                       int32_t threads, momenti_motif* out, int32_t out_stride, int32_t* n_out,
                       momenti_stats* stats, int32_t* rc, char* err, int32_t err_len) {
  if (err && err_len > 0) err[0] = 0;
  if (B < 0 || out_stride < 0) return MOMENTI_ERR_ARG;
  if (B == 0) return MOMENTI_OK;
  if (!params || !series || !dtype || !n || !D || !out || !n_out) return MOMENTI_ERR_ARG;
  for (int32_t b = 0; b < B; ++b)
    if (params[b].k > out_stride) return MOMENTI_ERR_ARG;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return MOMENTI_ERR_CUDA;
  // longest first (n * D windows to hash), so the tail of the batch is short
  std::vector<int32_t> order(static_cast<size_t>(B));
  for (int32_t b = 0; b < B; ++b) order[size_t(b)] = b;
  std::stable_sort(order.begin(), order.end(), [&](int32_t x, int32_t y) {
    return double(n[x]) * D[x] > double(n[y]) * D[y];
  });
  int T = threads > 0 ? threads : 8;
  if (T > B) T = B;
  // a zero memory limit shares 80% of the free memory among the workers
  size_t free_b = 0, total_b = 0;
  if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) return MOMENTI_ERR_CUDA;
  const uint64_t share = uint64_t(0.8 * double(free_b) / T);
  // a series nobody finished (a worker that could not start) reports an error
  std::vector<int> status(size_t(B), MOMENTI_ERR_CUDA);
  std::vector<std::string> messages(static_cast<size_t>(B));
  std::atomic<int32_t> next{0};
  // several workers: their exact-path sweeps share persistent launches
  std::unique_ptr<SweepBatcher> batcher;
  if (T > 1) batcher.reset(new (std::nothrow) SweepBatcher(T));
  auto worker = [&]() {
    cudaSetDevice(dev);
    struct Done {                   // leaves the batcher on every exit
      SweepBatcher* b;
      ~Done() {
        if (b) b->worker_done();
      }
    } done{batcher.get()};
    momenti_handle* h = new (std::nothrow) momenti_handle();
    if (!h) return;
    h->batcher = batcher.get();
    bool stream_ok = cudaStreamCreateWithFlags(&h->own_stream, cudaStreamNonBlocking) == cudaSuccess;
    for (;;) {
      const int32_t q = next.fetch_add(1);
      if (q >= B) break;
      const int32_t b = order[size_t(q)];
      int r = MOMENTI_ERR_CUDA;
      n_out[b] = 0;
      momenti_handle* probe = nullptr;
      if (!stream_ok) {
        fail(h, MOMENTI_ERR_CUDA, "topk_batch: cannot create a stream");
      } else if ((r = momenti_create(&probe, &params[b])) == MOMENTI_OK) {
        momenti_destroy(probe);
        h->p = params[b];
        if (h->p.mem_limit == 0) h->p.mem_limit = share;
        r = momenti_hash_all(h, series[b], dtype[b], n[b], D[b], n[b], on_device, h->own_stream);
        if (r == MOMENTI_OK)
          r = momenti_topk(h, out + int64_t(b) * out_stride, n_out + b, stats ? stats + b : nullptr);
      } else {
        fail(h, r, "topk_batch: invalid parameters");
      }
      status[size_t(b)] = r;
      if (r != MOMENTI_OK) {
        try {
          messages[size_t(b)] = h->err;
        } catch (...) {                 // the status alone still reports the failure
        }
      }
    }
    momenti_destroy(h);
  };
  std::vector<std::thread> pool;
  for (int t = 1; t < T; ++t) {
    try {
      pool.emplace_back(worker);
    } catch (...) {
      // fewer workers: the others take the rest (and the batcher stops
      // waiting for the ones that never started)
      for (int u = t; u < T; ++u)
        if (batcher) batcher->worker_done();
      break;
    }
  }
  worker();
  for (auto& th : pool) th.join();
  int first = MOMENTI_OK;
  for (int32_t b = 0; b < B; ++b) {
    if (rc) rc[b] = status[size_t(b)];
    if (first == MOMENTI_OK && status[size_t(b)] != MOMENTI_OK) {
      first = status[size_t(b)];
      if (err && err_len > 0)
        std::snprintf(err, size_t(err_len), "series %d: %s", int(b), messages[size_t(b)].c_str());
    }
  }
  return first;
}

int momenti_verify(momenti_handle* h, const int64_t* pairs, int64_t m, double* per_dim,
                   double* dist_d, uint64_t* dims_mask, int32_t fp64) {
  if (!h) return MOMENTI_ERR_ARG;
  if (!h->ready) return fail(h, MOMENTI_ERR_STATE, "verify before hash_all");
  if (m < 0 || (m > 0 && !pairs)) return fail(h, MOMENTI_ERR_ARG, "verify: bad pairs");
  if (m == 0) return MOMENTI_OK;
  const Index& ix = h->ix;
  std::vector<uint64_t> pk(m);
  for (int64_t q = 0; q < m; ++q) {
    int64_t a = pairs[2 * q], b = pairs[2 * q + 1];
    if (a < 0 || b < 0 || a >= ix.M || b >= ix.M) return fail(h, MOMENTI_ERR_ARG, "verify: index outside [0, M)");
    pk[q] = (uint64_t(a) << 32) | uint64_t(b);
  }
  cudaStream_t s = h->stream;
  uint64_t* dp = nullptr;
  double *dpd = nullptr, *ddd = nullptr;
  uint64_t* dmask = nullptr;
  CK(pool_malloc(&dp, m * 8, s));
  CK(pool_malloc(&dpd, m * ix.D * 8, s));
  CK(pool_malloc(&ddd, m * 8, s));
  CK(pool_malloc(&dmask, m * 8, s));
  CK(cudaMemcpyAsync(dp, pk.data(), m * 8, cudaMemcpyHostToDevice, s));
  CK(launch_verify_pairs(ix, h->p.d, dp, m, fp64, dpd, ddd, dmask, s));
  if (per_dim) CK(cudaMemcpyAsync(per_dim, dpd, m * ix.D * 8, cudaMemcpyDeviceToHost, s));
  if (dist_d) CK(cudaMemcpyAsync(dist_d, ddd, m * 8, cudaMemcpyDeviceToHost, s));
  if (dims_mask) CK(cudaMemcpyAsync(dims_mask, dmask, m * 8, cudaMemcpyDeviceToHost, s));
  CK(cudaFreeAsync(dp, s));
  CK(cudaFreeAsync(dpd, s));
  CK(cudaFreeAsync(ddd, s));
  CK(cudaFreeAsync(dmask, s));
  CK(cudaStreamSynchronize(s));
  return MOMENTI_OK;
}

int momenti_get_info(const momenti_handle* h, int64_t* M, int32_t* D, int32_t* L, int32_t* K,
                     double* r) {
  if (!h) return MOMENTI_ERR_ARG;
  if (!h->ready) return MOMENTI_ERR_STATE;
  if (M) *M = h->ix.M;
  if (D) *D = h->ix.D;
  if (L) *L = h->ix.L;
  if (K) *K = h->ix.K;
  if (r) *r = h->ix.r;
  return MOMENTI_OK;
}

int momenti_get_window_stats(momenti_handle* h, double* mu, double* sigma) {
  if (!h) return MOMENTI_ERR_ARG;
  if (!h->ready) return fail(h, MOMENTI_ERR_STATE, "get_window_stats before hash_all");
  const size_t cnt = size_t(h->ix.D) * h->ix.M;
  if (mu) CK(cudaMemcpyAsync(mu, h->ix.mu, cnt * 8, cudaMemcpyDeviceToHost, h->stream));
  if (sigma) CK(cudaMemcpyAsync(sigma, h->ix.sig, cnt * 8, cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  return MOMENTI_OK;
}

int momenti_get_keys(momenti_handle* h, int32_t j, uint64_t* keys) {
  if (!h) return MOMENTI_ERR_ARG;
  if (!h->ready) return fail(h, MOMENTI_ERR_STATE, "get_keys before hash_all");
  if (!keys || j < 0 || j >= h->ix.L) return fail(h, MOMENTI_ERR_ARG, "get_keys: bad arguments");
  const size_t cnt = size_t(h->ix.D) * h->ix.M;
  CK(cudaMemcpyAsync(keys, h->ix.keys + size_t(j) * cnt, cnt * 8, cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  return MOMENTI_OK;
}

int momenti_get_hash_draws(momenti_handle* h, float* a, float* u) {
  if (!h) return MOMENTI_ERR_ARG;
  if (!h->ready) return fail(h, MOMENTI_ERR_STATE, "get_hash_draws before hash_all");
  if (!a && !u) return fail(h, MOMENTI_ERR_ARG, "get_hash_draws: no output");
  const Index& ix = h->ix;
  // the device copies hold L_src repetitions per dim (L_src = L_used for
  // device draws, the supplied count for set_hash_params): copy the first L_used
  const bool tens = (h->p.flags & MOMENTI_FLAG_TENSORING) != 0;
  const int n_fn = tens ? 2 * isqrt(ix.L) : ix.L, K_fn = tens ? ix.K / 2 : ix.K;
  const int L_src = h->user_a.empty() ? n_fn : h->user_L;
  const size_t ra = size_t(n_fn) * K_fn * ix.w, rs = size_t(L_src) * K_fn * ix.w;
  const size_t ua = size_t(n_fn) * K_fn, us = size_t(L_src) * K_fn;
  if (a) CK(cudaMemcpy2DAsync(a, ra * 4, h->draw_a, rs * 4, ra * 4, ix.D, cudaMemcpyDeviceToHost, h->stream));
  if (u) CK(cudaMemcpy2DAsync(u, ua * 4, h->draw_u, us * 4, ua * 4, ix.D, cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  return MOMENTI_OK;
}

int momenti_get_index(momenti_handle* h, int32_t j, int32_t f, uint32_t* order, uint8_t* lcp) {
  if (!h) return MOMENTI_ERR_ARG;
  if (!h->ready) return fail(h, MOMENTI_ERR_STATE, "get_index before hash_all");
  if (j < 0 || j >= h->ix.L || f < 0 || f >= h->ix.D) return fail(h, MOMENTI_ERR_ARG, "get_index: bad (j, f)");
  const size_t off = (size_t(j) * h->ix.D + f) * h->ix.M;
  if (order) CK(cudaMemcpyAsync(order, h->ix.order + off, h->ix.M * 4, cudaMemcpyDeviceToHost, h->stream));
  if (lcp) CK(cudaMemcpyAsync(lcp, h->ix.lcp + off, h->ix.M, cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  return MOMENTI_OK;
}

int momenti_collide(momenti_handle* h, int32_t i, int32_t j, int64_t* pairs, int64_t cap,
                    int64_t* count) {
  if (!h) return MOMENTI_ERR_ARG;
  if (!h->ready) return fail(h, MOMENTI_ERR_STATE, "collide before hash_all");
  if (i < 1 || i > h->ix.K || j < 0 || j >= h->ix.L || cap < 0 || !count || (cap > 0 && !pairs))
    return fail(h, MOMENTI_ERR_ARG, "collide: bad arguments");
  cudaStream_t s = h->stream;
  uint64_t* dout = nullptr;
  const uint64_t dcap = uint64_t(std::max<int64_t>(cap, 1));
  CK(pool_malloc(&dout, dcap * 8, s));
  CK(cudaMemsetAsync(h->cs.counters, 0, 8 * sizeof(unsigned long long), s));
  CK(launch_collide(h->ix, i, j, j + 1, h->p.d, h->hs, h->cs, 1, dout, uint64_t(cap), s));
  unsigned long long c = 0;
  CK(cudaMemcpyAsync(&c, h->cs.counters, 8, cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  const int64_t got = std::min<int64_t>(int64_t(c), cap);
  std::vector<uint64_t> tmp(got);
  if (got) CK(cudaMemcpyAsync(tmp.data(), dout, got * 8, cudaMemcpyDeviceToHost, s));
  CK(cudaFreeAsync(dout, s));
  CK(cudaStreamSynchronize(s));
  for (int64_t q = 0; q < got; ++q) {
    pairs[2 * q] = int64_t(tmp[q] >> 32);
    pairs[2 * q + 1] = int64_t(tmp[q] & 0xffffffffu);
  }
  *count = int64_t(c);
  return MOMENTI_OK;
}


// ---- entry points: no C++ exception crosses the ABI ----

int momenti_create(momenti_handle** out, const momenti_params* p) {
  try {
    return create_impl(out, p);
  } catch (const std::bad_alloc&) {
    return fail(nullptr, MOMENTI_ERR_MEMORY, "host memory exhausted");
  } catch (...) {
    return fail(nullptr, MOMENTI_ERR_CUDA, "unexpected internal error");
  }
}

int momenti_set_hash_params(momenti_handle* h, int32_t D, int32_t L, int32_t K, int32_t w,
                            const float* a, const float* u) {
  try {
    return set_hash_params_impl(h, D, L, K, w, a, u);
  } catch (const std::bad_alloc&) {
    return fail(h, MOMENTI_ERR_MEMORY, "host memory exhausted");
  } catch (...) {
    return fail(h, MOMENTI_ERR_CUDA, "unexpected internal error");
  }
}

int momenti_hash_all(momenti_handle* h, const void* series, int32_t dtype, int64_t n, int32_t D,
                     int64_t ld, int32_t on_device, void* stream) {
  try {
    return hash_all_impl(h, series, dtype, n, D, ld, on_device, stream);
  } catch (const std::bad_alloc&) {
    return fail(h, MOMENTI_ERR_MEMORY, "host memory exhausted");
  } catch (...) {
    return fail(h, MOMENTI_ERR_CUDA, "unexpected internal error");
  }
}

int momenti_topk(momenti_handle* h, momenti_motif* out, int32_t* n_out, momenti_stats* stats) {
  try {
    return topk_impl(h, out, n_out, stats);
  } catch (const std::bad_alloc&) {
    return fail(h, MOMENTI_ERR_MEMORY, "host memory exhausted");
  } catch (...) {
    return fail(h, MOMENTI_ERR_CUDA, "unexpected internal error");
  }
}

int momenti_search_begin(momenti_handle* h, int32_t d_low, int32_t d_high) {
  try {
    return search_begin_impl(h, d_low, d_high);
  } catch (const std::bad_alloc&) {
    return fail(h, MOMENTI_ERR_MEMORY, "host memory exhausted");
  } catch (...) {
    return fail(h, MOMENTI_ERR_CUDA, "unexpected internal error");
  }
}

int momenti_search_step(momenti_handle* h, int64_t max_reps, int32_t* ended) {
  try {
    if (max_reps < 1) return fail(h, MOMENTI_ERR_ARG, "search_step: max_reps < 1");
    return search_step_impl(h, max_reps, ended);
  } catch (const std::bad_alloc&) {
    return fail(h, MOMENTI_ERR_MEMORY, "host memory exhausted");
  } catch (...) {
    return fail(h, MOMENTI_ERR_CUDA, "unexpected internal error");
  }
}

int momenti_search_current(momenti_handle* h, momenti_motif* out, int32_t* n_out, int32_t* cursor) {
  try {
    return search_current_impl(h, out, n_out, cursor);
  } catch (...) {
    return fail(h, MOMENTI_ERR_CUDA, "unexpected internal error");
  }
}

int momenti_search_finish(momenti_handle* h, momenti_motif* out, int32_t* n_out, int32_t* stops,
                          momenti_stats* stats) {
  try {
    return search_finish_impl(h, out, n_out, stops, stats);
  } catch (const std::bad_alloc&) {
    return fail(h, MOMENTI_ERR_MEMORY, "host memory exhausted");
  } catch (...) {
    return fail(h, MOMENTI_ERR_CUDA, "unexpected internal error");
  }
}

int momenti_topk_multi(momenti_handle* h, int32_t d_low, int32_t d_high, momenti_motif* out,
                       int32_t* n_out, int32_t* stops, momenti_stats* stats) {
  try {
    return topk_core(h, d_low, d_high, out, n_out, stops, stats);
  } catch (const std::bad_alloc&) {
    return fail(h, MOMENTI_ERR_MEMORY, "host memory exhausted");
  } catch (...) {
    return fail(h, MOMENTI_ERR_CUDA, "unexpected internal error");
  }
}

int momenti_topk_exact(momenti_handle* h, momenti_motif* out, int32_t* n_out) {
  try {
    return topk_exact_impl(h, out, n_out);
  } catch (const std::bad_alloc&) {
    return fail(h, MOMENTI_ERR_MEMORY, "host memory exhausted");
  } catch (...) {
    return fail(h, MOMENTI_ERR_CUDA, "unexpected internal error");
  }
}

int momenti_topk_batch(int32_t B, const momenti_params* params, const void* const* series,
                       const int32_t* dtype, const int64_t* n, const int32_t* D, int32_t on_device,
                       int32_t threads, momenti_motif* out, int32_t out_stride, int32_t* n_out,
                       momenti_stats* stats, int32_t* rc, char* err, int32_t err_len) {
  try {
    return topk_batch_impl(B, params, series, dtype, n, D, on_device, threads, out, out_stride, n_out, stats, rc, err, err_len);
  } catch (const std::bad_alloc&) {
    return fail(nullptr, MOMENTI_ERR_MEMORY, "host memory exhausted");
  } catch (...) {
    return fail(nullptr, MOMENTI_ERR_CUDA, "unexpected internal error");
  }
}

// ---- host arithmetic of the search, callable without a device ----

double momenti_collision_probability(double R, double r) {
  if (!(r > 0.0) || std::isnan(R)) return std::nan("");
  return collision_probability(R, r);
}

double momenti_failure_bound(double dist_max, int32_t i, int32_t j, int32_t K, int32_t L,
                             int32_t d, double r) {
  if (K < 1 || i < 1 || i > K || j < 0 || j > L || d < 1 || !(r > 0.0) || std::isnan(dist_max))
    return std::nan("");
  return failure_bound(dist_max, i, j, K, L, d, r);
}

// Miss probability of a pair under tensoring after j repetitions at prefix
// length i (Section 6.1, bound re-derived): L = m^2 repetitions, repetition
// j' (0-based) pairs left function j' div m with right function j' mod m,
// keys interleave their K/2 values (left first), so length t needs the
// left prefix ceil(t/2) and the right prefix floor(t/2) to collide.  Each
// value collides independently with probability p, so a function's
// collision depth G has P(G >= u) = p^u.  Rows (left functions) and
// columns (right functions) fall into groups visited alike; the largest
// depth class of each group decides the miss, and the sum runs over them.
double momenti_tensoring_failure_bound(double p, int32_t i, int32_t j, int32_t K, int32_t L) {
  if (!(p >= 0.0 && p <= 1.0) || K < 2 || K % 2 || i < 1 || i > K || L < 1 || j < 0 || j > L)
    return std::nan("");
  int32_t m = 0;
  while (int64_t(m + 1) * (m + 1) <= L) ++m;
  if (m * m != L) return std::nan("");
  const bool top = i == K;
  const int ug0 = (i + 1) / 2, ug1 = top ? ug0 : (i + 2) / 2;   // ceil(i/2), ceil((i+1)/2)
  const int uh0 = i / 2, uh1 = top ? uh0 : (i + 1) / 2;         // floor(i/2), floor((i+1)/2)
  // largest class among n iid functions: -1 (none) or 0, 1, 2
  auto max_class = [&](int u0, int u1, int64_t n, double out[4]) {
    const double s1 = std::pow(p, u0), s2 = std::pow(p, u1);
    const double cdf[3] = {1.0 - s1, 1.0 - s2, 1.0};
    for (int c = 0; c < 4; ++c) out[c] = 0.0;
    if (n == 0) {
      out[0] = 1.0;                                                // class -1 at index 0
      return;
    }
    double prev = 0.0;
    for (int c = 0; c < 3; ++c) {
      const double cur = std::pow(std::min(1.0, cdf[c]), double(n));
      out[c + 1] = cur - prev;
      prev = cur;
    }
  };
  const int64_t a = j / m, b = j % m;
  const int64_t rows[3] = {a, a < m ? 1 : 0, std::max<int64_t>(0, m - a - 1)};
  const int64_t cols[2] = {b, m - b};
  // (row group, column group, 0: length i / 1: length i + 1)
  int visits[6][3] = {{0, 0, 0}, {0, 1, 0}, {1, 0, 0}, {1, 1, 1}, {2, 0, 1}, {2, 1, 1}};
  const int nv = top ? 3 : 6;
  double g[3][4], hc[2][4];
  for (int q = 0; q < 3; ++q) max_class(ug0, ug1, rows[q], g[q]);
  for (int q = 0; q < 2; ++q) max_class(uh0, uh1, cols[q], hc[q]);
  double miss = 0.0;
  int gm[3], hm[2];
  for (gm[0] = 0; gm[0] < 4; ++gm[0])
    for (gm[1] = 0; gm[1] < 4; ++gm[1])
      for (gm[2] = 0; gm[2] < 4; ++gm[2])
        for (hm[0] = 0; hm[0] < 4; ++hm[0])
          for (hm[1] = 0; hm[1] < 4; ++hm[1]) {
            const double pr = g[0][gm[0]] * g[1][gm[1]] * g[2][gm[2]] * hc[0][hm[0]] * hc[1][hm[1]];
            if (pr == 0.0) continue;
            bool hit = false;
            for (int v = 0; v < nv && !hit; ++v) {
              // stored index = class + 1; a visit at length i needs class >= 1
              // on both sides, at length i + 1 class 2
              const int need = 2 + visits[v][2];
              hit = gm[visits[v][0]] >= need && hm[visits[v][1]] >= need;
            }
            if (!hit) miss += pr;
          }
  return miss;
}

static int top_select_impl(const float* dd, const int64_t* a, const int64_t* b, int64_t m,
                           int32_t k, int64_t eps, int64_t batch, int64_t* idx, int32_t* n_out) {
  if (m < 0 || k < 1 || eps < 0 || batch < 1 || !idx || !n_out) return MOMENTI_ERR_ARG;
  if (m > 0 && (!dd || !a || !b)) return MOMENTI_ERR_ARG;
  *n_out = 0;
  std::vector<PairRec> rec(static_cast<size_t>(m));
  std::unordered_map<uint64_t, int64_t> first;     // pair -> first position
  for (int64_t q = 0; q < m; ++q) {
    if (std::isnan(dd[q]) || a[q] < 0 || b[q] <= a[q] || b[q] > int64_t(UINT32_MAX))
      return MOMENTI_ERR_ARG;
    PairRec& r = rec[size_t(q)];
    r = PairRec{};
    r.a = uint32_t(a[q]);
    r.b = uint32_t(b[q]);
    r.dist_d = dd[q];
    r.dist_max = dd[q];
    first.emplace((uint64_t(r.a) << 32) | r.b, q);
  }
  Pool pool;
  pool.k = k;
  pool.eps = eps;
  for (int64_t q0 = 0; q0 < m; q0 += batch)
    pool.add(rec.data() + q0, size_t(std::min<int64_t>(batch, m - q0)));
  int32_t n = 0;
  for (const PoolEntry& e : pool.top) idx[n++] = first.at((uint64_t(e.a) << 32) | e.b);
  *n_out = n;
  return MOMENTI_OK;
}

int momenti_top_select(const float* dd, const int64_t* a, const int64_t* b, int64_t m,
                       int32_t k, int64_t eps, int64_t batch, int64_t* idx, int32_t* n_out) {
  try {
    return top_select_impl(dd, a, b, m, k, eps, batch, idx, n_out);
  } catch (const std::bad_alloc&) {
    return fail(nullptr, MOMENTI_ERR_MEMORY, "host memory exhausted");
  } catch (...) {
    return fail(nullptr, MOMENTI_ERR_CUDA, "unexpected internal error");
  }
}
}  // extern "C"
