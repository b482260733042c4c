// The row-minima form of the wide all-pairs sweep at 64 dims
// (k_allpairs_rows2<64, true>, defined in k_verify_kernels.cuh), in a
// translation unit of its own so that it compiles in parallel with the
// others.
#include "k_verify_kernels.cuh"

namespace momenti {

cudaError_t launch_rows2_64_rowmin(const Index& ix, int d, float* rowmin, cudaStream_t s) {
  return rows2_dispatch<64, true>(ix, d, 0.f, ApRec{}, rowmin, s);
}

}  // namespace momenti
