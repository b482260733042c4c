// Allocation-free variant of the index sort (the per-(repetition, dim)
// sort of hash keys that momenti_hash_all runs), for callers that must not
// allocate device memory.  The paper has no counterpart.
//
// Its scratch (two ping-pong key/index buffers, the digit histograms and
// the partition's work lists) is one file-scope __device__ array of fixed
// size, so the entry point
// never calls cudaMalloc, cudaFree or any allocating routine.  In host code
// the array's name is only a stand-in for the symbol: its device address
// is looked up with cudaGetSymbolAddress (with the device current) and that
// address is what the kernels receive.  The address belongs to the CUDA
// context the module was loaded into, so it is cached per device together
// with that context's unique id and looked up again whenever the current
// context differs (after cudaDeviceReset, for instance, the module is
// loaded again into a new primary context and the array may move).
#include "../../include/momenti.h"
#include "internal.h"

#include <cuda.h>

#include <mutex>

namespace {

constexpr int64_t kMaxKeys = MOMENTI_NOALLOC_MAX_KEYS;
constexpr size_t kBytes = momenti::sort_scratch_bytes(kMaxKeys, 1);

// Shared by every call on a device; keeps the last call's contents.
static __device__ __align__(256) unsigned char g_sort_scratch[kBytes];

constexpr int kMaxDevices = 64;
struct Slot {
  unsigned long long ctx_id = 0;   // unique id of the context the address belongs to
  unsigned char* addr = nullptr;
};
std::mutex g_mu;
Slot g_slot[kMaxDevices];

// Unique id of the calling thread's current context (driver entry points
// fetched through the runtime, so the library needs no link to libcuda);
// 0 when there is none or the driver cannot tell.
unsigned long long current_ctx_id() {
  using GetCurrent = CUresult (*)(CUcontext*);
  using GetId = CUresult (*)(CUcontext, unsigned long long*);
  static GetCurrent get_current = nullptr;
  static GetId get_id = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q{};
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess && q == cudaDriverEntryPointSuccess)
      get_current = reinterpret_cast<GetCurrent>(p);
    p = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess && q == cudaDriverEntryPointSuccess)
      get_id = reinterpret_cast<GetId>(p);
  });
  if (!get_current || !get_id) return 0;
  CUcontext c = nullptr;
  if (get_current(&c) != CUDA_SUCCESS || !c) return 0;
  unsigned long long id = 0;
  if (get_id(c, &id) != CUDA_SUCCESS) return 0;
  return id;
}

}  // namespace

extern "C" int momenti_index_sort_noalloc(const uint64_t* keys, int64_t m, int32_t K,
                                          uint32_t* order, uint8_t* lcp, void* stream) {
  if (m < 0 || K < 1 || K > MOMENTI_MAX_K) return MOMENTI_ERR_ARG;
  if (m > kMaxKeys) return MOMENTI_ERR_OVERFLOW;     // beyond the fixed scratch
  if (m == 0) return MOMENTI_OK;
  if (!keys || !order || !lcp) return MOMENTI_ERR_ARG;
  // an error left pending by earlier work of the caller is reported, not
  // cleared, and is not mixed up with this call's own launches
  if (cudaPeekAtLastError() != cudaSuccess) return MOMENTI_ERR_CUDA;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return MOMENTI_ERR_CUDA;
  unsigned char* base = nullptr;
  {
    std::lock_guard<std::mutex> lk(g_mu);
    Slot& sl = g_slot[dev];
    unsigned long long id = current_ctx_id();
    if (!sl.addr || id == 0 || id != sl.ctx_id) {
      void* p = nullptr;
      if (cudaGetSymbolAddress(&p, g_sort_scratch) != cudaSuccess || !p) {
        sl = Slot{};
        return MOMENTI_ERR_CUDA;
      }
      if (id == 0) id = current_ctx_id();   // the lookup made the primary context current
      sl.ctx_id = id;                       // 0: looked up again on every call
      sl.addr = static_cast<unsigned char*>(p);
    }
    base = sl.addr;
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
  // every level is launched with fixed grids (no host round trip, no pinned
  // buffer); the kernels stop at the work counts they find on the device
  momenti::SortScratch sc = momenti::sort_scratch_carve(base, kMaxKeys, 1);
  sc.M = m;
  sc.caps = momenti::sort_caps(m, 1);
  cudaError_t e = momenti::launch_sort_reps(ix, 0, 1, sc, static_cast<cudaStream_t>(stream));
  return e == cudaSuccess ? MOMENTI_OK : MOMENTI_ERR_CUDA;
}
