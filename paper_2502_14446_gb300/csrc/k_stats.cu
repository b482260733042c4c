// Series layout, rolling window statistics, the r heuristic and the hash
// functions of Eq. (drp).
//
// Window statistics follow Eq. (zned): mean and population standard
// deviation of every length-w window, from float64 running sums of
// (x - c) and (x - c)^2 with Neumaier compensation, c being the first value
// of a block of consecutive windows (restarting the sums every block keeps
// the rounding drift bounded).  Where the variance from the sums has lost
// more than nine digits to cancellation (a near-constant window), the
// window is recomputed by the two-pass formula, which gives exactly 0 for a
// constant window.  A window is flat when sigma <= 1e-8 (1 + |mu|); its
// z-normalised form is the zero vector.
#include "internal.h"

#include <cmath>

namespace momenti {

namespace {

__global__ void k_split_f32(const float* __restrict__ src, int64_t n, int D, int64_t ld,
                            float* __restrict__ hi) {
  int64_t total = int64_t(D) * n;
  for (int64_t q = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; q < total;
       q += int64_t(gridDim.x) * blockDim.x) {
    int64_t f = q / n, t = q - f * n;
    hi[q] = src[f * ld + t];
  }
}

__global__ void k_split_f64(const double* __restrict__ src, int64_t n, int D, int64_t ld,
                            float* __restrict__ hi, float* __restrict__ lo) {
  int64_t total = int64_t(D) * n;
  for (int64_t q = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; q < total;
       q += int64_t(gridDim.x) * blockDim.x) {
    int64_t f = q / n, t = q - f * n;
    double x = src[f * ld + t];
    float h = float(x);
    hi[q] = h;
    lo[q] = float(x - double(h));
  }
}

struct Neumaier {
  double s = 0.0, c = 0.0;
  __device__ void add(double v) {
    double t = s + v;
    if (fabs(s) >= fabs(v)) c += (s - t) + v;
    else c += (v - t) + s;
    s = t;
  }
  __device__ double value() const { return s + c; }
};

constexpr int kStatsChunk = 64;

template <bool LO>
__global__ void k_window_stats(const float* __restrict__ xh, const float* __restrict__ xl,
                               int64_t n, int64_t M, int w, double* __restrict__ mu,
                               double* __restrict__ sig, float* __restrict__ mh,
                               float* __restrict__ ml, float* __restrict__ isg) {
  const int f = blockIdx.y;
  const int64_t a0 = (blockIdx.x * int64_t(blockDim.x) + threadIdx.x) * kStatsChunk;
  if (a0 >= M) return;
  const int64_t a1 = min(M, a0 + kStatsChunk);
  const float* xf = xh + int64_t(f) * n;
  const float* lf = LO ? xl + int64_t(f) * n : nullptr;
  auto X = [&](int64_t t) -> double {
    double v = double(xf[t]);
    if (LO) v += double(lf[t]);
    return v;
  };
  const double c = X(a0);
  Neumaier s1, s2;
  for (int t = 0; t < w; ++t) {
    double y = X(a0 + t) - c;
    s1.add(y);
    s2.add(y * y);
  }
  const double inv_w = 1.0 / double(w);
  for (int64_t a = a0; a < a1; ++a) {
    if (a > a0) {
      double yo = X(a - 1) - c, yi = X(a + w - 1) - c;
      s1.add(-yo);
      s1.add(yi);
      s2.add(-yo * yo);
      s2.add(yi * yi);
    }
    double m1 = s1.value() * inv_w;
    double m2 = s2.value() * inv_w;
    double var = m2 - m1 * m1;
    double mean = c + m1;
    if (!(var > 1e-9 * m2)) {
      // cancellation ate most digits (near-constant window): two passes
      double s = 0.0;
      for (int t = 0; t < w; ++t) s += X(a + t);
      mean = s * inv_w;
      double q = 0.0;
      for (int t = 0; t < w; ++t) {
        double y = X(a + t) - mean;
        q += y * y;
      }
      var = q * inv_w;
    }
    double sd = sqrt(var);
    bool flat = sd <= kFlatRel * (1.0 + fabs(mean));
    int64_t o = int64_t(f) * M + a;
    mu[o] = mean;
    sig[o] = sd;
    float hi = float(mean);
    mh[o] = hi;
    ml[o] = float(mean - double(hi));
    isg[o] = flat ? 0.f : float(1.0 / sd);
  }
}

__device__ inline void atomic_min_f(float* p, float v) {
  int* ip = reinterpret_cast<int*>(p);
  int old = *ip;
  while (__int_as_float(old) > v) {
    int prev = atomicCAS(ip, old, __float_as_int(v));
    if (prev == old) break;
    old = prev;
  }
}
__device__ inline void atomic_max_f(float* p, float v) {
  int* ip = reinterpret_cast<int*>(p);
  int old = *ip;
  while (__int_as_float(old) < v) {
    int prev = atomicCAS(ip, old, __float_as_int(v));
    if (prev == old) break;
    old = prev;
  }
}

// One thread per (sample window, dim): the z-normalised window projected on
// the K vectors of repetition 0; block min/max then one atomic per block.
__global__ void k_r_sample(const float* __restrict__ xh, const float* __restrict__ xl,
                           const float* __restrict__ mh, const float* __restrict__ ml,
                           const float* __restrict__ isg, const float* __restrict__ a32,
                           int64_t n, int64_t M, int w, int Wp, int N, int K, int S,
                           float* __restrict__ out2) {
  const int f = blockIdx.y;
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  float lo = INFINITY, hi = -INFINITY;
  if (q < S) {
    int64_t a = (S <= 1) ? 0 : (int64_t(q) * (M - 1)) / (S - 1);
    int64_t o = int64_t(f) * M + a;
    const float m0 = mh[o], m1 = ml[o], is = isg[o];
    const float* x = xh + int64_t(f) * n + a;
    const float* xlo = xl ? xl + int64_t(f) * n + a : nullptr;
    const float* A = a32 + int64_t(f) * Wp * N;
    float acc[kRepStride];
#pragma unroll
    for (int k = 0; k < kRepStride; ++k) acc[k] = 0.f;
    for (int t = 0; t < w; ++t) {
      float z = (x[t] - m0) + ((xlo ? xlo[t] : 0.f) - m1);
#pragma unroll
      for (int k = 0; k < kRepStride; ++k) acc[k] = fmaf(A[int64_t(t) * N + k], z, acc[k]);
    }
    for (int k = 0; k < K; ++k) {
      float v = acc[k] * is;
      lo = fminf(lo, v);
      hi = fmaxf(hi, v);
    }
  }
  for (int off = 16; off > 0; off >>= 1) {
    lo = fminf(lo, __shfl_xor_sync(0xffffffffu, lo, off));
    hi = fmaxf(hi, __shfl_xor_sync(0xffffffffu, hi, off));
  }
  __shared__ float slo[32], shi[32];
  int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) { slo[wid] = lo; shi[wid] = hi; }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int i = 1; i < int(blockDim.x >> 5); ++i) { lo = fminf(lo, slo[i]); hi = fmaxf(hi, shi[i]); }
    atomic_min_f(out2, lo);
    atomic_max_f(out2 + 1, hi);
  }
}

// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11), as published.
struct Philox {
  __device__ static inline void round(uint32_t c[4], uint32_t k[2]) {
    const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
    uint32_t hi0 = __umulhi(M0, c[0]), lo0 = M0 * c[0];
    uint32_t hi1 = __umulhi(M1, c[2]), lo1 = M1 * c[2];
    uint32_t n0 = hi1 ^ c[1] ^ k[0], n2 = hi0 ^ c[3] ^ k[1];
    c[0] = n0; c[1] = lo1; c[2] = n2; c[3] = lo0;
  }
  __device__ static inline void gen(uint64_t seed, uint64_t ctr, uint32_t stream, uint32_t out[4]) {
    uint32_t c[4] = {uint32_t(ctr), uint32_t(ctr >> 32), stream, 0u};
    uint32_t k[2] = {uint32_t(seed), uint32_t(seed >> 32)};
    for (int r = 0; r < 10; ++r) {
      round(c, k);
      k[0] += 0x9E3779B9u;
      k[1] += 0xBB67AE85u;
    }
    out[0] = c[0]; out[1] = c[1]; out[2] = c[2]; out[3] = c[3];
  }
};

__device__ inline float u01_open_closed(uint32_t x) { return float((x >> 8) + 1u) * 5.9604645e-8f; }
__device__ inline float u01(uint32_t x) { return float(x >> 8) * 5.9604645e-8f; }

// a: count_a normals (Box-Muller on Philox outputs, stream 0), rounded to
// half; u: count_u uniforms in [0, 1) (stream 1).
__global__ void k_draw(uint64_t seed, int64_t count_a, int64_t count_u, float* __restrict__ a,
                       float* __restrict__ u) {
  int64_t g = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  int64_t stride = int64_t(gridDim.x) * blockDim.x;
  for (int64_t q = g; q * 4 < count_a; q += stride) {
    uint32_t r[4];
    Philox::gen(seed, uint64_t(q), 0u, r);
    float z[4];
    for (int h = 0; h < 2; ++h) {
      float u1 = u01_open_closed(r[2 * h]), u2 = u01(r[2 * h + 1]);
      float rad = sqrtf(-2.f * logf(u1));
      float s, c;
      sincospif(2.f * u2, &s, &c);
      z[2 * h] = rad * c;
      z[2 * h + 1] = rad * s;
    }
    for (int e = 0; e < 4; ++e) {
      int64_t o = q * 4 + e;
      if (o < count_a) a[o] = __half2float(__float2half_rn(z[e]));
    }
  }
  for (int64_t q = g; q * 4 < count_u; q += stride) {
    uint32_t r[4];
    Philox::gen(seed, uint64_t(q), 1u, r);
    for (int e = 0; e < 4; ++e) {
      int64_t o = q * 4 + e;
      if (o < count_u) u[o] = u01(r[e]);
    }
  }
}

__global__ void k_layout_hash(const float* __restrict__ a_src, int D, int L, int L_src, int K,
                              int w, int Wp, __half* __restrict__ a16, float* __restrict__ a32) {
  const int N = L * kRepStride;
  int64_t total = int64_t(D) * N * Wp;
  for (int64_t q = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; q < total;
       q += int64_t(gridDim.x) * blockDim.x) {
    int64_t f = q / (int64_t(N) * Wp);
    int64_t rem = q - f * N * Wp;
    int nn = int(rem / Wp), t = int(rem - int64_t(nn) * Wp);
    int j = nn / kRepStride, kk = nn - j * kRepStride;
    float v = 0.f;
    if (kk < K && t < w) v = a_src[((f * L_src + j) * K + kk) * w + t];
    a16[q] = __float2half_rn(v);
    a32[(f * Wp + t) * N + nn] = __half2float(__float2half_rn(v));
  }
}

__global__ void k_layout_boff(const float* __restrict__ u_src, int D, int L, int L_src, int K,
                              double r, float* __restrict__ boff) {
  const int N = L * kRepStride;
  int64_t total = int64_t(D) * N;
  for (int64_t q = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; q < total;
       q += int64_t(gridDim.x) * blockDim.x) {
    int64_t f = q / N;
    int nn = int(q - f * N);
    int j = nn / kRepStride, kk = nn - j * kRepStride;
    float b = 0.f;
    if (kk < K) b = float(double(u_src[(f * L_src + j) * K + kk]) * r);
    boff[q] = b;
  }
}

__global__ void k_point_major(const float* __restrict__ hi, const float* __restrict__ lo,
                              int64_t n, int D, int Dp, float* __restrict__ xT,
                              float* __restrict__ xlT) {
  const int64_t total = n * Dp;
  for (int64_t q = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; q < total;
       q += int64_t(gridDim.x) * blockDim.x) {
    const int64_t t = q / Dp;
    const int f = int(q - t * Dp);
    xT[q] = f < D ? hi[int64_t(f) * n + t] : 0.f;
    if (lo) xlT[q] = f < D ? lo[int64_t(f) * n + t] : 0.f;
  }
}

// Means of 16 consecutive points, point-major, from float64 running sums
// restarted every 256 points.
__global__ void k_mean16(const float* __restrict__ hi, const float* __restrict__ lo, int64_t n,
                         int D, int Dp, float* __restrict__ smT) {
  const int f = blockIdx.y;
  const int64_t t0 = (blockIdx.x * int64_t(blockDim.x) + threadIdx.x) * 256;
  const int64_t m = n - 15;
  if (t0 >= m) return;
  const int64_t t1 = min(m, t0 + 256);
  const float* x = hi + int64_t(f) * n;
  const float* y = lo ? lo + int64_t(f) * n : nullptr;
  auto X = [&](int64_t t) { return double(x[t]) + (y ? double(y[t]) : 0.0); };
  double s = 0.0;
  for (int u = 0; u < 16; ++u) s += X(t0 + u);
  for (int64_t t = t0; t < t1; ++t) {
    if (t > t0) s += X(t + 15) - X(t - 1);
    smT[t * Dp + f] = float(s * (1.0 / 16.0));
  }
}

__global__ void k_stats_pm(const float* __restrict__ mh, const float* __restrict__ ml,
                           const float* __restrict__ isg, int64_t M, int D, int Dp,
                           float* __restrict__ stT) {
  const int64_t total = M * Dp;
  for (int64_t q = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; q < total;
       q += int64_t(gridDim.x) * blockDim.x) {
    const int64_t a = q / Dp;
    const int f = int(q - a * Dp);
    const int64_t o = int64_t(f) * M + a;
    float* dst = stT + a * 3 * Dp;
    dst[f] = f < D ? mh[o] : 0.f;
    dst[Dp + f] = f < D ? ml[o] : 0.f;
    dst[2 * Dp + f] = f < D ? isg[o] : 0.f;
  }
}

inline int grid_for(int64_t work, int block) {
  int64_t g = (work + block - 1) / block;
  if (g > sm_count() * 32) g = sm_count() * 32;
  if (g < 1) g = 1;
  return int(g);
}

}  // namespace

cudaError_t launch_split_series(const void* src, int dtype, int64_t n, int D, int64_t ld,
                                float* hi, float* lo, cudaStream_t s) {
  int g = grid_for(int64_t(D) * n, 256);
  if (dtype == 0)
    MOMENTI_LAUNCH("split_f32", s, k_split_f32<<<g, 256, 0, s>>>(static_cast<const float*>(src), n, D, ld, hi));
  else
    MOMENTI_LAUNCH("split_f64", s, k_split_f64<<<g, 256, 0, s>>>(static_cast<const double*>(src), n, D, ld, hi, lo));
  return cudaGetLastError();
}

cudaError_t launch_window_stats(const Index& ix, cudaStream_t s) {
  int64_t chunks = (ix.M + kStatsChunk - 1) / kStatsChunk;
  dim3 grid(unsigned((chunks + 127) / 128), unsigned(ix.D));
  if (ix.has_lo)
    MOMENTI_LAUNCH("window_stats", s, k_window_stats<true><<<grid, 128, 0, s>>>(ix.xs_hi, ix.xs_lo, ix.n, ix.M, ix.w, ix.mu, ix.sig,
                                              ix.mu_hi, ix.mu_lo, ix.inv_sig));
  else
    MOMENTI_LAUNCH("window_stats", s, k_window_stats<false><<<grid, 128, 0, s>>>(ix.xs_hi, nullptr, ix.n, ix.M, ix.w, ix.mu, ix.sig,
                                               ix.mu_hi, ix.mu_lo, ix.inv_sig));
  return cudaGetLastError();
}

cudaError_t launch_point_major(const Index& ix, cudaStream_t s) {
  if (ix.xW)
    MOMENTI_LAUNCH("point_major", s, k_point_major<<<grid_for(ix.n * ix.DW, 256), 256, 0, s>>>(ix.xs_hi, nullptr, ix.n, ix.D, ix.DW, ix.xW, nullptr));
  if (!ix.xT) return cudaGetLastError();
  MOMENTI_LAUNCH("point_major", s, k_point_major<<<grid_for(ix.n * ix.Dp, 256), 256, 0, s>>>(ix.xs_hi, ix.has_lo ? ix.xs_lo : nullptr, ix.n, ix.D, ix.Dp, ix.xT, ix.xlT));
  if (ix.smT) {
    const int64_t chunks = (ix.n - 15 + 255) / 256;
    dim3 grid{unsigned((chunks + 127) / 128), unsigned(ix.D), 1u};
    MOMENTI_LAUNCH("mean16", s, k_mean16<<<grid, 128, 0, s>>>(ix.xs_hi, ix.has_lo ? ix.xs_lo : nullptr, ix.n, ix.D, ix.Dp, ix.smT));
  }
  return cudaGetLastError();
}

cudaError_t launch_stats_point_major(const Index& ix, cudaStream_t s) {
  if (!ix.stT) return cudaSuccess;
  MOMENTI_LAUNCH("stats_pm", s, k_stats_pm<<<grid_for(ix.M * ix.Dp, 256), 256, 0, s>>>(ix.mu_hi, ix.mu_lo, ix.inv_sig, ix.M, ix.D, ix.Dp, ix.stT));
  return cudaGetLastError();
}

cudaError_t launch_r_sample(const Index& ix, int S, float* out2, cudaStream_t s) {
  dim3 grid(unsigned((S + 127) / 128), unsigned(ix.D));
  MOMENTI_LAUNCH("r_sample", s, k_r_sample<<<grid, 128, 0, s>>>(ix.xs_hi, ix.has_lo ? ix.xs_lo : nullptr, ix.mu_hi, ix.mu_lo,
                                  ix.inv_sig, ix.a32, ix.n, ix.M, ix.w, ix.Wp, ix.L * kRepStride,
                                  ix.K, S, out2));
  return cudaGetLastError();
}

cudaError_t launch_draw_hash(uint64_t seed, int D, int L, int K, int w, float* a_out,
                             float* u_out, cudaStream_t s) {
  int64_t ca = int64_t(D) * L * K * w, cu = int64_t(D) * L * K;
  MOMENTI_LAUNCH("draw", 0, k_draw<<<grid_for((ca + 3) / 4, 256), 256, 0, s>>>(seed, ca, cu, a_out, u_out));
  return cudaGetLastError();
}

cudaError_t launch_layout_hash(const Index& ix, const float* a_src, int L_src, cudaStream_t s) {
  int64_t total = int64_t(ix.D) * ix.L * kRepStride * ix.Wp;
  MOMENTI_LAUNCH("layout_hash", 0, k_layout_hash<<<grid_for(total, 256), 256, 0, s>>>(a_src, ix.D, ix.L, L_src, ix.K, ix.w, ix.Wp,
                                                      ix.a16, ix.a32));
  return cudaGetLastError();
}

cudaError_t launch_layout_boff(const Index& ix, const float* u_src, int L_src, cudaStream_t s) {
  int64_t total = int64_t(ix.D) * ix.L * kRepStride;
  MOMENTI_LAUNCH("layout_boff", 0, k_layout_boff<<<grid_for(total, 256), 256, 0, s>>>(u_src, ix.D, ix.L, L_src, ix.K, ix.r, ix.boff));
  return cudaGetLastError();
}

}  // namespace momenti
