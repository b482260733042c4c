// The statistics form of the wide all-pairs sweep at 64 dims
// (k_allpairs_rows4<64>, defined in k_verify_kernels.cuh) in a translation
// unit of its own: the 64-dimension instantiations are the slowest part of
// the library to compile, and translation units compile in parallel.
#include "k_verify_kernels.cuh"

namespace momenti {

cudaError_t launch_rows4_64(const Index& ix, int d, float thr, const ApRec& rc, cudaStream_t s,
                            int64_t gy_max) {
  return rows4_launch<64>(ix, d, thr, rc, s, gy_max);
}

}  // namespace momenti
