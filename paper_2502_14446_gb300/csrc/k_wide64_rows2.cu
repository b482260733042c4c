// The slid form of the wide all-pairs sweep at 64 dims, recording pairs
// (k_allpairs_rows2<64, false>, defined in k_verify_kernels.cuh), in a
// translation unit of its own so that it compiles in parallel with the
// others.
#include "k_verify_kernels.cuh"

namespace momenti {

cudaError_t launch_rows2_64(const Index& ix, int d, float thr, const ApRec& rc, cudaStream_t s,
                            int64_t gy_max) {
  return rows2_launch<64>(ix, d, thr, rc, s, gy_max);
}

}  // namespace momenti
