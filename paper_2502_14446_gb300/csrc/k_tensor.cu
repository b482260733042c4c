// Tensoring (Section 6.1): composite keys of the m^2 repetitions from the
// keys of 2 m half functions of K/2 hash values each.  Repetition j'
// (0-based) takes left function l = j' div m (half index 2 l) and right
// function r = j' mod m (half index 2 r + 1) and interleaves their values,
// a left value first: hash value 2 q is the left value q and 2 q + 1 the
// right value q.  The half keys hold their K/2 values in the leading bytes
// (the packing of every composite key), so the interleave is one byte
// permutation per 32-bit half of the result.
#include "internal.h"

#include <algorithm>

namespace momenti {

namespace {

__global__ void k_tensor_keys(const uint64_t* __restrict__ half, int64_t M, int D, int m,
                              int j0, int j1, uint64_t* __restrict__ keys) {
  const int64_t per_rep = M * D;
  const int64_t total = int64_t(j1 - j0) * per_rep;
  for (int64_t q = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; q < total;
       q += int64_t(gridDim.x) * blockDim.x) {
    const int64_t jr = q / per_rep, e = q - jr * per_rep;   // e = a * D + f
    const int j = j0 + int(jr);
    const int l = j / m, r = j - (j / m) * m;
    const uint32_t lw = uint32_t(half[int64_t(2 * l) * per_rep + e] >> 32);
    const uint32_t rw = uint32_t(half[int64_t(2 * r + 1) * per_rep + e] >> 32);
    // bytes (most significant first) L0 R0 L1 R1 | L2 R2 L3 R3
    const uint32_t hi = __byte_perm(lw, rw, 0x3726u);
    const uint32_t lo = __byte_perm(lw, rw, 0x1504u);
    keys[int64_t(j) * per_rep + e] = (uint64_t(hi) << 32) | lo;
  }
}

}  // namespace

cudaError_t launch_tensor_keys(const Index& ix, const uint64_t* half, int m, int j0, int j1,
                               cudaStream_t s) {
  if (j1 <= j0) return cudaSuccess;
  const int64_t total = int64_t(j1 - j0) * ix.M * ix.D;
  const int g = int(std::min<int64_t>((total + 255) / 256, int64_t(sm_count()) * 16));
  MOMENTI_LAUNCH("tensor_keys", s, k_tensor_keys<<<g, 256, 0, s>>>(half, ix.M, ix.D, m, j0, j1, ix.keys));
  return cudaGetLastError();
}

}  // namespace momenti
