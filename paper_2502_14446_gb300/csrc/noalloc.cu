// Allocation-free variant of the index sort (the per-(repetition, dim)
// sort of hash keys that momenti_hash_all runs), for callers that must not
// allocate device memory.  The paper has no counterpart.
//
// Its scratch (two ping-pong key/index buffers and the digit histograms)
// is one file-scope __device__ array of fixed size, so the entry point
// never calls cudaMalloc, cudaFree or any allocating routine.  In host code
// the array's name is only a stand-in for the symbol: its device address
// is looked up once per device with cudaGetSymbolAddress (with that device
// current, on the first call made on it) and that address is what the
// kernels receive.
#include "../../include/momenti.h"
#include "internal.h"

#include <mutex>

namespace {

constexpr int64_t kMaxKeys = MOMENTI_NOALLOC_MAX_KEYS;
constexpr int64_t kTile = 2048;   // entries per CTA of the sort kernels
constexpr int64_t kHistEntries = 256 * ((kMaxKeys + kTile - 1) / kTile);
constexpr size_t kBytes = size_t(kMaxKeys) * (8 + 8 + 4 + 4) + size_t(kHistEntries) * 4;

// Shared by every call on a device; keeps the last call's contents.
static __device__ __align__(256) unsigned char g_sort_scratch[kBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
unsigned char* g_addr[kMaxDevices] = {};

}  // namespace

extern "C" int momenti_index_sort_noalloc(const uint64_t* keys, int64_t m, int32_t K,
                                          uint32_t* order, uint8_t* lcp, void* stream) {
  if (m < 0 || K < 1 || K > MOMENTI_MAX_K) return MOMENTI_ERR_ARG;
  if (m > kMaxKeys) return MOMENTI_ERR_OVERFLOW;     // beyond the fixed scratch
  if (m == 0) return MOMENTI_OK;
  if (!keys || !order || !lcp) return MOMENTI_ERR_ARG;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return MOMENTI_ERR_CUDA;
  unsigned char* base = nullptr;
  {
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_addr[dev]) {
      void* p = nullptr;
      if (cudaGetSymbolAddress(&p, g_sort_scratch) != cudaSuccess || !p) return MOMENTI_ERR_CUDA;
      g_addr[dev] = static_cast<unsigned char*>(p);
    }
    base = g_addr[dev];
  }
  momenti::Index ix;
  ix.M = m;
  ix.n = m;
  ix.D = 1;
  ix.K = K;
  ix.L = 1;
  ix.keys = const_cast<uint64_t*>(keys);
  ix.order = order;
  ix.lcp = lcp;
  momenti::SortScratch sc;
  sc.k0 = reinterpret_cast<uint64_t*>(base);
  sc.k1 = sc.k0 + kMaxKeys;
  sc.v0 = reinterpret_cast<uint32_t*>(sc.k1 + kMaxKeys);
  sc.v1 = sc.v0 + kMaxKeys;
  sc.hist = sc.v1 + kMaxKeys;
  sc.cap_entries = kMaxKeys;
  sc.hist_entries = kHistEntries;
  cudaError_t e = momenti::launch_sort_reps(ix, 0, 1, sc, static_cast<cudaStream_t>(stream));
  return e == cudaSuccess ? MOMENTI_OK : MOMENTI_ERR_CUDA;
}
