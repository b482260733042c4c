// Launch accounting and optional per-kernel event timing.  Every kernel
// launch of the library passes through prof_begin / prof_end: a process-wide
// counter, and, for the one kernel selected by momenti_time_kernel, a pair
// of CUDA events recorded on the launching stream around the launch.
#include "../../include/momenti.h"
#include "internal.h"

#include <atomic>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

namespace momenti {
namespace {
std::atomic<uint64_t> g_launches{0};
std::mutex g_mu;
std::string g_name;
struct Ev { cudaEvent_t a, b; };
std::vector<Ev> g_pending;
std::vector<Ev> g_pool;
double g_ms = 0.0;
uint64_t g_count = 0;
bool g_on = false;

Ev take_ev() {
  if (!g_pool.empty()) { Ev e = g_pool.back(); g_pool.pop_back(); return e; }
  Ev e;
  cudaEventCreate(&e.a);
  cudaEventCreate(&e.b);
  return e;
}
thread_local Ev t_cur{nullptr, nullptr};
thread_local bool t_timing = false;
}  // namespace

int sm_count() {
  static std::atomic<int> cache[64] = {};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 1;
  int c = cache[dev].load(std::memory_order_relaxed);
  if (c > 0) return c;
  if (cudaDeviceGetAttribute(&c, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || c < 1) c = 1;
  cache[dev].store(c, std::memory_order_relaxed);
  return c;
}

cudaError_t allow_smem(const void* func, size_t bytes) {
  static std::mutex mu;
  static std::map<std::pair<int, const void*>, size_t> granted;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lk(mu);
  size_t& g = granted[{dev, func}];
  if (bytes <= g) return cudaSuccess;
  e = cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, int(bytes));
  if (e == cudaSuccess) g = bytes;
  return e;
}

void prof_begin(const char* name, cudaStream_t s) {
  g_launches.fetch_add(1, std::memory_order_relaxed);
  if (!g_on) return;
  std::lock_guard<std::mutex> lk(g_mu);
  // "prefix*" selects every kernel whose name starts with prefix
  const size_t n = g_name.size();
  const bool match = (n > 0 && g_name[n - 1] == '*') ? std::strncmp(g_name.c_str(), name, n - 1) == 0
                                                    : g_name == name;
  if (!match) return;
  t_cur = take_ev();
  t_timing = true;
  cudaEventRecord(t_cur.a, s);
}

void prof_end(const char* name, cudaStream_t s) {
  (void)name;
  if (!t_timing) return;
  t_timing = false;
  cudaEventRecord(t_cur.b, s);
  std::lock_guard<std::mutex> lk(g_mu);
  g_pending.push_back(t_cur);
}

}  // namespace momenti

using namespace momenti;

extern "C" {

uint64_t momenti_launch_count(void) { return g_launches.load(); }

int momenti_time_kernel(const char* name) {
  std::lock_guard<std::mutex> lk(g_mu);
  for (auto& e : g_pending) g_pool.push_back(e);
  g_pending.clear();
  g_ms = 0.0;
  g_count = 0;
  g_on = name != nullptr;
  g_name = name ? name : "";
  return MOMENTI_OK;
}

int momenti_kernel_time(double* total_ms, uint64_t* launches) {
  std::lock_guard<std::mutex> lk(g_mu);
  for (auto& e : g_pending) {
    if (cudaEventSynchronize(e.b) != cudaSuccess) return MOMENTI_ERR_CUDA;
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e.a, e.b);
    g_ms += ms;
    ++g_count;
    g_pool.push_back(e);
  }
  g_pending.clear();
  if (total_ms) *total_ms = g_ms;
  if (launches) *launches = g_count;
  return MOMENTI_OK;
}

}  // extern "C"
