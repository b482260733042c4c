// Plain FP32 form of the projections and hashes of Algorithm 1 (its hashing step):
// h_{K,j}^f(T_a) = floor((a . z_a + b) / r) (Eq. drp) for every window a,
// dimension f and repetition j, packed into one 64-bit key per (j, a, f).
//
// Canonical FP32 arithmetic (shared with the tensor-core path's rehash, so
// that both forms give the same key bits):
//   z_t = (xh[a+t] - mu_hi[a]) + (xl[a+t] - mu_lo[a])
//   acc = fma(a_t, z_t, acc) for t = 0 .. w-1 in order, acc = 0 initially
//   v   = acc * inv_sigma[a]                (v = a . z_a, z-normalised)
//   q   = (v + b) * inv_r
//   h   = clamp(floor(q), -128, 127); byte = h + 128
// and the key holds byte k at bits 56 - 8k (big-endian: the prefix of
// length i is the top 8i bits, Section 4's lexicographic order).
//
// Tiling: a CTA computes 64 windows x 8 repetitions (64 projections) of one
// dimension; the series segment and the projection vectors of each t-chunk
// are staged in shared memory.  Thread (tw, tr) owns windows tw and tw+32
// and repetition tr, i.e. 2 x 8 accumulators.
#include "internal.h"

namespace momenti {

namespace {

constexpr int kBM = 64;    // windows per CTA
constexpr int kBR = 8;     // repetitions per CTA
constexpr int kBN = kBR * kRepStride;
constexpr int kTK = 32;    // t-chunk

__device__ __forceinline__ uint32_t hash_byte(float acc, float isg, float b, float inv_r) {
  float v = acc * isg;
  float q = (v + b) * inv_r;
  float h = floorf(q);
  h = fminf(fmaxf(h, -128.f), 127.f);
  return uint32_t(int(h) + 128);
}

template <bool LO>
__global__ void __launch_bounds__(256)
k_proj_hash_fp32(const float* __restrict__ xh, const float* __restrict__ xl,
                 const float* __restrict__ mh, const float* __restrict__ ml,
                 const float* __restrict__ isg, const float* __restrict__ a32,
                 const float* __restrict__ boff, float inv_r, int64_t n, int64_t M, int D,
                 int w, int Wp, int N, int K, int j0, int j1, uint64_t* __restrict__ keys) {
  __shared__ float sx[kBM + kTK];
  __shared__ float sxl[LO ? kBM + kTK : 1];
  __shared__ __align__(16) float sb[kTK][kBN];

  // dims fastest: the D CTAs of a window tile store into the same key rows
  const int f = int(blockIdx.x % unsigned(D));
  const int64_t a0 = int64_t(blockIdx.x / unsigned(D)) * kBM;
  const int jb = j0 + blockIdx.y * kBR;
  const int tid = threadIdx.x;
  const int tw = tid & 31, tr = tid >> 5;

  const float* xf = xh + int64_t(f) * n;
  const float* lf = LO ? xl + int64_t(f) * n : nullptr;
  const float* Af = a32 + int64_t(f) * Wp * N;

  int64_t wa[2] = {a0 + tw, a0 + tw + 32};
  float m0[2], m1[2];
  for (int u = 0; u < 2; ++u) {
    int64_t o = int64_t(f) * M + (wa[u] < M ? wa[u] : 0);
    m0[u] = mh[o];
    m1[u] = ml[o];
  }
  float acc[2][kRepStride];
#pragma unroll
  for (int u = 0; u < 2; ++u)
#pragma unroll
    for (int k = 0; k < kRepStride; ++k) acc[u][k] = 0.f;

  const int nb0 = jb * kRepStride;
  for (int t0 = 0; t0 < w; t0 += kTK) {
    __syncthreads();
    for (int q = tid; q < kBM + kTK; q += blockDim.x) {
      int64_t p = a0 + t0 + q;
      sx[q] = p < n ? xf[p] : 0.f;
      if (LO) sxl[q] = p < n ? lf[p] : 0.f;
    }
    for (int q = tid; q < kTK * kBN; q += blockDim.x) {
      int tt = q / kBN, c = q - tt * kBN;
      int t = t0 + tt, nn = nb0 + c;
      sb[tt][c] = (t < Wp && nn < N) ? Af[int64_t(t) * N + nn] : 0.f;
    }
    __syncthreads();
    const int tmax = min(kTK, w - t0);
    for (int tt = 0; tt < tmax; ++tt) {
      float z0 = (sx[tw + tt] - m0[0]) + ((LO ? sxl[tw + tt] : 0.f) - m1[0]);
      float z1 = (sx[tw + 32 + tt] - m0[1]) + ((LO ? sxl[tw + 32 + tt] : 0.f) - m1[1]);
      const float4 b0 = *reinterpret_cast<const float4*>(&sb[tt][tr * kRepStride]);
      const float4 b1 = *reinterpret_cast<const float4*>(&sb[tt][tr * kRepStride + 4]);
      const float bv[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
      for (int k = 0; k < kRepStride; ++k) {
        acc[0][k] = fmaf(bv[k], z0, acc[0][k]);
        acc[1][k] = fmaf(bv[k], z1, acc[1][k]);
      }
    }
  }

  const int j = jb + tr;
  if (j >= j1) return;
  const float* bo = boff + int64_t(f) * N + int64_t(j) * kRepStride;
  float bvals[kRepStride];
#pragma unroll
  for (int k = 0; k < kRepStride; ++k) bvals[k] = bo[k];
  for (int u = 0; u < 2; ++u) {
    if (wa[u] >= M) continue;
    const float is = isg[int64_t(f) * M + wa[u]];
    uint64_t key = 0;
#pragma unroll
    for (int k = 0; k < kRepStride; ++k) {
      uint64_t byte = (k < K) ? hash_byte(acc[u][k], is, bvals[k], inv_r) : 0u;
      key |= byte << (56 - 8 * k);
    }
    keys[(int64_t(j) * M + wa[u]) * D + f] = key;
  }
}

}  // namespace

cudaError_t launch_proj_hash_fp32(const Index& ix, int j0, int j1, cudaStream_t s) {
  if (j1 <= j0) return cudaSuccess;
  dim3 grid(unsigned(ix.D * ((ix.M + kBM - 1) / kBM)), unsigned((j1 - j0 + kBR - 1) / kBR), 1u);
  const int N = ix.L * kRepStride;
  if (ix.has_lo)
    MOMENTI_LAUNCH("proj_hash_fp32", s, k_proj_hash_fp32<true><<<grid, 256, 0, s>>>(ix.xs_hi, ix.xs_lo, ix.mu_hi, ix.mu_lo, ix.inv_sig,
                                                ix.a32, ix.boff, ix.inv_r, ix.n, ix.M, ix.D, ix.w,
                                                ix.Wp, N, ix.K, j0, j1, ix.keys));
  else
    MOMENTI_LAUNCH("proj_hash_fp32", s, k_proj_hash_fp32<false><<<grid, 256, 0, s>>>(ix.xs_hi, nullptr, ix.mu_hi, ix.mu_lo, ix.inv_sig,
                                                 ix.a32, ix.boff, ix.inv_r, ix.n, ix.M, ix.D, ix.w,
                                                 ix.Wp, N, ix.K, j0, j1, ix.keys));
  return cudaGetLastError();
}

}  // namespace momenti
