// The per-step-load all-pairs sweep at 64 dims (k_allpairs_wide<64>,
// defined in k_verify_kernels.cuh: series without a point-major copy, e.g.
// float64 input with 32 < D <= 64), both forms, in a translation unit of
// its own so that it compiles in parallel with the others.
#include "k_verify_kernels.cuh"

namespace momenti {

namespace {

template <bool ROWMIN>
cudaError_t wide64(const Index& ix, int d, float thr, const ApRec& rc, float* rowmin, cudaStream_t s) {
  const int64_t ndiag = ix.M - (ix.excl + 1);
  if (ndiag <= 0) return cudaSuccess;
  const int64_t gy = (ndiag + kDiagBlock - 1) / kDiagBlock;
  const size_t smem = size_t(64) * (kDiagBlock + 1) * sizeof(float);
  cudaError_t e = allow_smem(reinterpret_cast<const void*>(k_allpairs_wide<64, ROWMIN>), smem);
  if (e != cudaSuccess) return e;
  for (int64_t y0 = 0; y0 < gy; y0 += 65535) {
    dim3 grid{unsigned((ix.M + kSeg - 1) / kSeg), unsigned(std::min<int64_t>(65535, gy - y0)), 1u};
    MOMENTI_LAUNCH("allpairs", s, k_allpairs_wide<64, ROWMIN><<<grid, kDiagBlock, smem, s>>>(ix, d, thr, rc, rowmin, y0));
  }
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_wide64(const Index& ix, int d, float thr, const ApRec& rc, float* rowmin,
                          bool rowmin_mode, cudaStream_t s) {
  return rowmin_mode ? wide64<true>(ix, d, thr, rc, rowmin, s) : wide64<false>(ix, d, thr, rc, rowmin, s);
}

}  // namespace momenti
