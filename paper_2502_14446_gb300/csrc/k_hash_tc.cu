// Tensor-core form of the projections and hashes of Algorithm 1 (its hashing step)
// (Eq. drp on z-normalised windows), for sm_103a: tcgen05.mma with TMEM
// accumulators, projection vectors staged by TMA.
//
// Per CTA: one dimension f and 128 consecutive windows (the TMEM lanes).
// The product is Z (128 x w, the z-normalised Hankel rows of the series) by
// the projection vectors (w x N, N = 8 per repetition).  Z never exists in
// global memory: converter warps build each 128 x 64 K-chunk of it in shared
// memory from the raw series segment and the window statistics, in the
// 128-byte-swizzled K-major layout the MMA reads, as two half-precision
// operands z = z_hi + z_lo (z_hi = half(z), z_lo = half(z - z_hi)); the
// product accumulates z_hi . a + z_lo . a in FP32, so it is exact to about
// 2^-22 relative (the vectors a are half-representable by construction).
//
// Warp roles (26 warps): 0 TMA producer of the vectors, 1 MMA issuer and
// TMEM owner, 2-9 converters (two threads per row, half a K-chunk each),
// 10-25 epilogue (four warps per TMEM lane quarter, a quarter of the
// columns each).  A 3-stage ring of
// (Z_hi, Z_lo, vectors) chunks feeds the MMA; two 256-column TMEM
// accumulators let the epilogue hash one 32-repetition block while the next
// one is multiplied.  Every wait is bounded: on timeout the kernel raises
// an error flag the host reads, drains its own copies and frees TMEM.
//
// Epilogue: q = (v + b) / r, h = clamp(floor(q), -128, 127).  A value with
// |q - round(q)| < 2^-11 is flagged; the rehash kernel recomputes flagged
// values with the canonical FP32 arithmetic of the CUDA-core form, so both
// forms produce the same key bits.
#include "internal.h"

#include <cuda.h>

namespace momenti {

namespace {

constexpr int kBM = 128;
constexpr int kBN = 256;                 // projections per TMEM accumulator (32 reps)
constexpr int kBK = 64;                  // fp16 per 128-byte swizzle row
constexpr int kStages = 3;
constexpr int kAStage = kBM * kBK * 2;   // 16 KB per operand half
constexpr int kBStage = kBN * kBK * 2;   // 32 KB
constexpr int kConvWarps = 8;
constexpr int kEpiWarps = 16;
constexpr int kThreads = 32 * (2 + kConvWarps + kEpiWarps);
constexpr float kMargin = 1.0f / 2048.0f;
constexpr long long kSpinCycles = 4000000000ll;   // about 2 s at 2 GHz

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return uint32_t(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool mbar_try(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      "selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}
// Bounded wait: false (and the error flag raised) on timeout or when
// another role already failed.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, int* err) {
  long long t0 = clock64();
  int it = 0;
  while (!mbar_try(bar, parity)) {
    if ((++it & 255) == 0) {
      if (*reinterpret_cast<volatile int*>(err)) return false;
      if (clock64() - t0 > kSpinCycles) {
        atomicOr(err, 1);
        return false;
      }
    }
  }
  return true;
}

__device__ __forceinline__ void fence_proxy_async() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

// UMMA shared-memory descriptor: K-major, 128-byte swizzle, 8-row groups
// 1024 bytes apart.
__device__ __forceinline__ uint64_t sdesc(uint32_t addr) {
  uint64_t d = 0;
  d |= uint64_t((addr & 0x3FFFF) >> 4);          // start address
  d |= uint64_t(1) << 16;                        // leading byte offset (unused for SW128 K-major)
  d |= uint64_t(1024 >> 4) << 32;                // stride byte offset
  d |= uint64_t(1) << 46;                        // descriptor version
  d |= uint64_t(2) << 61;                        // SWIZZLE_128B
  return d;
}

// Instruction descriptor, kind::f16: F16 x F16 -> F32, both K-major.
constexpr uint32_t kIdesc = (1u << 4) | (0u << 7) | (0u << 10) | (uint32_t(kBN >> 3) << 17) |
                            (uint32_t(kBM >> 4) << 24);

__device__ __forceinline__ void umma(uint32_t dtmem, uint64_t a, uint64_t b, uint32_t acc) {
  asm volatile(
      "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(dtmem),
      "l"(a), "l"(b), "r"(kIdesc), "r"(acc)
      : "memory");
}
__device__ __forceinline__ void umma_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
               : "memory");
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32]) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
      "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
      "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]),
        "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]),
        "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int q = 0; q < 32; ++q) v[q] = __uint_as_float(r[q]);
}

__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap* map, int x, int y,
                                            uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(bar)
      : "memory");
}

struct TcArgs {
  const float* xh;
  const float* xl;
  const float* mh;
  const float* ml;
  const float* isg;
  const float* boff;
  float inv_r;
  int64_t n, M;
  int D, w, Wp, N, K, L, j0, j1;
  uint64_t* keys;
  uint64_t* flags;
  uint32_t flag_cap;
  uint32_t* flag_count;
  int* err;
};

struct Smem {
  uint32_t a, b, x, st, bar, tslot;
  int seg;   // floats in the series segment
};

__device__ __forceinline__ Smem layout(uint8_t* base, int Wp, bool lo) {
  Smem s;
  const uint32_t b0 = smem_u32(base);
  s.a = b0;
  s.b = b0 + kStages * 2 * kAStage;
  s.x = s.b + kStages * kBStage;
  s.seg = kBM + Wp;
  s.st = s.x + s.seg * 4 * (lo ? 2 : 1);
  s.bar = (s.st + kBM * 12 + 7) & ~7u;
  s.tslot = s.bar + (3 * kStages + 5) * 8;
  return s;
}

__global__ void __launch_bounds__(kThreads, 1)
k_proj_hash_tc(const __grid_constant__ CUtensorMap tmap, TcArgs g) {
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  uint8_t* base = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  const bool lo = g.xl != nullptr;
  const Smem S = layout(base, g.Wp, lo);
  float* sx = reinterpret_cast<float*>(base + (S.x - smem_u32(base)));
  float* sxl = sx + S.seg;
  float* sst = reinterpret_cast<float*>(base + (S.st - smem_u32(base)));   // [3][128]
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  // the D dims of one window tile are neighbouring CTAs, so their 8-byte
  // key stores into the same [j][a][0..D) rows meet in L2
  const int f = int(blockIdx.x % unsigned(g.D));
  const int64_t a0 = int64_t(blockIdx.x / unsigned(g.D)) * kBM;
  const int KC = g.Wp / kBK;
  const int NC = (g.j1 - g.j0) * kRepStride;
  const int nchunks = (NC + kBN - 1) / kBN;
  const int steps = nchunks * KC;
  auto full_a = [&](int s) { return S.bar + 8u * s; };
  auto full_b = [&](int s) { return S.bar + 8u * (kStages + s); };
  auto empty = [&](int s) { return S.bar + 8u * (2 * kStages + s); };
  auto tfull = [&](int b) { return S.bar + 8u * (3 * kStages + b); };
  auto tempty = [&](int b) { return S.bar + 8u * (3 * kStages + 2 + b); };
  const uint32_t mma_done = S.bar + 8u * (3 * kStages + 4);

  // ---- set-up: series segment, window statistics, barriers, TMEM ----
  const float* xf = g.xh + int64_t(f) * g.n;
  const float* lf = lo ? g.xl + int64_t(f) * g.n : nullptr;
  for (int q = threadIdx.x; q < S.seg; q += kThreads) {
    int64_t p = a0 + q;
    sx[q] = p < g.n ? xf[p] : 0.f;
    if (lo) sxl[q] = p < g.n ? lf[p] : 0.f;
  }
  for (int q = threadIdx.x; q < kBM; q += kThreads) {
    int64_t a = a0 + q;
    bool v = a < g.M;
    int64_t o = int64_t(f) * g.M + (v ? a : 0);
    sst[q] = v ? g.mh[o] : 0.f;
    sst[kBM + q] = v ? g.ml[o] : 0.f;
    sst[2 * kBM + q] = v ? g.isg[o] : 0.f;
  }
  if (threadIdx.x == 0) {
    for (int s = 0; s < kStages; ++s) {
      mbar_init(full_a(s), kConvWarps);
      mbar_init(full_b(s), 1);
      mbar_init(empty(s), 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(tfull(b), 1);
      mbar_init(tempty(b), kEpiWarps);
    }
    mbar_init(mma_done, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    fence_proxy_async();
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 512;" ::"r"(S.tslot)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *reinterpret_cast<volatile uint32_t*>(base + (S.tslot - smem_u32(base)));

  if (warp == 0) {
    // ---- TMA producer: projection vectors ----
    if (lane == 0) {
      asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tmap)) : "memory");
      int issued = 0;
      for (int s = 0; s < steps; ++s) {
        const int st = s % kStages;
        if (s >= kStages && !mbar_wait(empty(st), ((s / kStages) - 1) & 1, g.err)) break;
        const int nc = s / KC, kc = s - nc * KC;
        mbar_expect_tx(full_b(st), kBStage);
        tma_load_2d(S.b + st * kBStage, &tmap, kc * kBK, f * g.N + g.j0 * kRepStride + nc * kBN,
                    full_b(st));
        issued = s + 1;
      }
      // drain: every issued copy has landed before the CTA may exit
      for (int s = (issued > kStages ? issued - kStages : 0); s < issued; ++s)
        mbar_wait(full_b(s % kStages), (s / kStages) & 1, g.err);
    }
  } else if (warp == 1) {
    // ---- MMA issuer ----
    if (lane == 0) {
      for (int nc = 0; nc < nchunks; ++nc) {
        const int buf = nc & 1;
        if (nc >= 2 && !mbar_wait(tempty(buf), ((nc >> 1) - 1) & 1, g.err)) break;
        tc_fence_after();
        const uint32_t dt = tmem + uint32_t(buf * kBN);
        bool ok = true;
        for (int kc = 0; kc < KC; ++kc) {
          const int s = nc * KC + kc, st = s % kStages, ph = (s / kStages) & 1;
          if (!mbar_wait(full_a(st), ph, g.err) || !mbar_wait(full_b(st), ph, g.err)) {
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t ahi = S.a + st * 2 * kAStage, alo = ahi + kAStage;
          const uint32_t bb = S.b + st * kBStage;
#pragma unroll
          for (int kk = 0; kk < kBK / 16; ++kk) {
            umma(dt, sdesc(ahi + kk * 32), sdesc(bb + kk * 32), (kc | kk) ? 1u : 0u);
            umma(dt, sdesc(alo + kk * 32), sdesc(bb + kk * 32), 1u);
          }
          umma_commit(empty(st));
        }
        if (!ok) break;
        umma_commit(tfull(buf));
      }
      // every MMA of this thread has completed before TMEM is released
      umma_commit(mma_done);
      mbar_wait(mma_done, 0, g.err);
    }
  } else if (warp < 2 + kConvWarps) {
    // ---- converters: z-normalised Hankel K-chunks, hi/lo halves ----
    const int ct = threadIdx.x - 64;
    const int m = ct >> 1;                          // row 0..127
    const int c0 = (ct & 1) * (kBK / 16);           // first of this thread's 16-byte chunks
    const float mh = sst[m], ml = sst[kBM + m], is = sst[2 * kBM + m];
    for (int s = 0; s < steps; ++s) {
      const int st = s % kStages;
      bool ok = s < kStages || mbar_wait(empty(st), ((s / kStages) - 1) & 1, g.err);
      if (!__all_sync(0xffffffffu, ok)) break;
      const int kc = s % KC;
      uint8_t* ahi = base + (S.a - smem_u32(base)) + st * 2 * kAStage;
      uint8_t* alo = ahi + kAStage;
#pragma unroll
      for (int cc = 0; cc < kBK / 16; ++cc) {
        const int c = c0 + cc;
        uint32_t hw[4], lw[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          const int t = kc * kBK + c * 8 + e * 2;
          float2 z;
          z.x = t < g.w ? ((sx[m + t] - mh) + ((lo ? sxl[m + t] : 0.f) - ml)) * is : 0.f;
          z.y = t + 1 < g.w ? ((sx[m + t + 1] - mh) + ((lo ? sxl[m + t + 1] : 0.f) - ml)) * is : 0.f;
          // packed conversions: hi = half(z), lo = half(z - hi)
          const __half2 h = __float22half2_rn(z);
          const float2 hb = __half22float2(h);
          const __half2 l = __float22half2_rn(make_float2(z.x - hb.x, z.y - hb.y));
          hw[e] = *reinterpret_cast<const uint32_t*>(&h);
          lw[e] = *reinterpret_cast<const uint32_t*>(&l);
        }
        const int chunk = c ^ (m & 7);
        *reinterpret_cast<uint4*>(ahi + m * 128 + chunk * 16) = make_uint4(hw[0], hw[1], hw[2], hw[3]);
        *reinterpret_cast<uint4*>(alo + m * 128 + chunk * 16) = make_uint4(lw[0], lw[1], lw[2], lw[3]);
      }
      fence_proxy_async();
      __syncwarp();
      if (lane == 0) mbar_arrive(full_a(st));
    }
  } else {
    // ---- epilogue: TMEM -> hash bytes -> keys ----
    const int ew = warp - (2 + kConvWarps);        // 0 .. kEpiWarps-1
    const int quarter = warp & 3;                  // TMEM lanes 32*quarter ..
    constexpr int kGroups = (kBN / 32) / (kEpiWarps / 4);   // column groups of 32 per warp
    const int qbeg = (ew >> 2) * kGroups, qend = qbeg + kGroups;
    const int m = quarter * 32 + lane;
    const int64_t a = a0 + m;
    const bool row_ok = a < g.M;
    const float* bo = g.boff + int64_t(f) * g.N + int64_t(g.j0) * kRepStride;
    for (int nc = 0; nc < nchunks; ++nc) {
      const int buf = nc & 1;
      bool ok = mbar_wait(tfull(buf), (nc >> 1) & 1, g.err);
      if (!__all_sync(0xffffffffu, ok)) break;
      tc_fence_after();
#pragma unroll 1
      for (int q = qbeg; q < qend; ++q) {
        // offsets of the 32 columns, scaled by 1/r, one per lane
        const int col0 = nc * kBN + q * 32;
        const float myb = col0 + lane < NC ? bo[col0 + lane] * g.inv_r : 0.f;
        float v[32];
        tmem_ld32(tmem + (uint32_t(quarter * 32) << 16) + uint32_t(buf * kBN + q * 32), v);
#pragma unroll
        for (int rr = 0; rr < 4; ++rr) {
          const int j = g.j0 + col0 / kRepStride + rr;
          const bool live = j < g.j1 && row_ok;      // warp-uniform in j, per lane in row
          uint64_t key = 0;
#pragma unroll
          for (int k = 0; k < kRepStride; ++k) {
            const float qv = fmaf(v[rr * 8 + k], g.inv_r, __shfl_sync(0xffffffffu, myb, rr * 8 + k));
            float h = floorf(qv);
            const float fr = qv - h;
            // near a bucket boundary: recomputed by the canonical FP32 form
            if (live && k < g.K && (fr < kMargin || fr > 1.f - kMargin)) {
              const uint32_t pos = atomicAdd(g.flag_count, 1u);
              const int nn = j * kRepStride + k;
              if (pos < g.flag_cap) g.flags[pos] = (uint64_t(f) << 56) | (uint64_t(nn) << 32) | uint64_t(a);
            }
            h = fminf(fmaxf(h, -128.f), 127.f);
            if (k < g.K) key |= uint64_t(int(h) + 128) << (56 - 8 * k);
          }
          if (live) g.keys[(int64_t(j) * g.M + a) * g.D + f] = key;
        }
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(tempty(buf));
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 512;" ::"r"(tmem) : "memory");
  }
}

// Canonical FP32 recomputation of flagged values (same arithmetic as the
// CUDA-core form): patches one byte of the key.
__global__ void k_rehash(const float* __restrict__ xh, const float* __restrict__ xl,
                         const float* __restrict__ mh, const float* __restrict__ ml,
                         const float* __restrict__ isg, const float* __restrict__ a32,
                         const float* __restrict__ boff, float inv_r, int64_t n, int64_t M, int D,
                         int w, int Wp, int N, const uint64_t* __restrict__ flags,
                         const uint32_t* __restrict__ count, uint32_t cap,
                         unsigned long long* __restrict__ keys) {
  uint32_t cnt = *count;
  if (cnt > cap) cnt = cap;
  for (uint32_t q = blockIdx.x * blockDim.x + threadIdx.x; q < cnt; q += gridDim.x * blockDim.x) {
    const uint64_t e = flags[q];
    const int f = int(e >> 56), nn = int((e >> 32) & 0xFFFFFFu);
    const int64_t a = int64_t(e & 0xFFFFFFFFu);
    const int64_t o = int64_t(f) * M + a;
    const float m0 = mh[o], m1 = ml[o], is = isg[o];
    const float* x = xh + int64_t(f) * n + a;
    const float* l = xl ? xl + int64_t(f) * n + a : nullptr;
    const float* A = a32 + int64_t(f) * Wp * N + nn;
    float acc = 0.f;
    for (int t = 0; t < w; ++t) {
      float z = (x[t] - m0) + ((l ? l[t] : 0.f) - m1);
      acc = fmaf(A[int64_t(t) * N], z, acc);
    }
    const float v = acc * is;
    const float qv = (v + boff[int64_t(f) * N + nn]) * inv_r;
    float h = floorf(qv);
    h = fminf(fmaxf(h, -128.f), 127.f);
    const int j = nn / kRepStride, k = nn % kRepStride;
    const int sh = 56 - 8 * k;
    unsigned long long* kp = keys + (int64_t(j) * M + a) * D + f;
    atomicAnd(kp, ~(0xFFull << sh));
    atomicOr(kp, uint64_t(int(h) + 128) << sh);
  }
}

using EncodeFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                              const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                              const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                              CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeFn encode_fn() {
  // initialised once, thread-safely (the batching form hashes from several threads)
  static const EncodeFn fn = []() -> EncodeFn {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      return reinterpret_cast<EncodeFn>(p);
    return nullptr;
  }();
  return fn;
}

size_t tc_smem_bytes(int Wp, bool lo) {
  size_t seg = size_t(kBM + Wp) * 4 * (lo ? 2 : 1);
  size_t bytes = size_t(kStages) * (2 * kAStage + kBStage) + seg + kBM * 12 + 8 + (3 * kStages + 5) * 8 + 16;
  return bytes + 1024;   // alignment slack
}

}  // namespace

bool tc_supported() {
  int dev = 0, major = 0, minor = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return false;
  cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev);
  cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev);
  return major == 10 && minor == 3 && encode_fn() != nullptr;
}

cudaError_t launch_proj_hash_tc(const Index& ix, int j0, int j1, uint64_t* flags, uint32_t flag_cap,
                                uint32_t* flag_count, int* err, cudaStream_t s) {
  if (j1 <= j0) return cudaSuccess;
  EncodeFn enc = encode_fn();
  if (!enc) return cudaErrorNotSupported;
  const int N = ix.L * kRepStride;
  CUtensorMap map;
  cuuint64_t gdim[2] = {cuuint64_t(ix.Wp), cuuint64_t(ix.D) * cuuint64_t(N)};
  cuuint64_t gstride[1] = {cuuint64_t(ix.Wp) * 2};
  cuuint32_t box[2] = {cuuint32_t(kBK), cuuint32_t(kBN)};
  cuuint32_t estride[2] = {1, 1};
  CUresult r = enc(&map, CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 2, ix.a16, gdim, gstride, box, estride,
                   CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                   CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return cudaErrorInvalidValue;
  TcArgs g{ix.xs_hi, ix.has_lo ? ix.xs_lo : nullptr, ix.mu_hi, ix.mu_lo, ix.inv_sig, ix.boff,
           ix.inv_r, ix.n, ix.M, ix.D, ix.w, ix.Wp, N, ix.K, ix.L, j0, j1, ix.keys, flags,
           flag_cap, flag_count, err};
  const size_t smem = tc_smem_bytes(ix.Wp, ix.has_lo);
  cudaError_t e = allow_smem(reinterpret_cast<const void*>(k_proj_hash_tc), smem);
  if (e != cudaSuccess) return e;
  dim3 grid{unsigned(ix.D * ((ix.M + kBM - 1) / kBM)), 1u, 1u};
  MOMENTI_LAUNCH("proj_hash_tc", s, k_proj_hash_tc<<<grid, kThreads, smem, s>>>(map, g));
  return cudaGetLastError();
}

cudaError_t launch_rehash_fp32(const Index& ix, const uint64_t* flags, const uint32_t* flag_count,
                               uint32_t flag_cap, cudaStream_t s) {
  MOMENTI_LAUNCH("rehash", s, k_rehash<<<sm_count() * 8, 256, 0, s>>>(ix.xs_hi, ix.has_lo ? ix.xs_lo : nullptr, ix.mu_hi, ix.mu_lo,
                                   ix.inv_sig, ix.a32, ix.boff, ix.inv_r, ix.n, ix.M, ix.D, ix.w,
                                   ix.Wp, ix.L * kRepStride, flags, flag_count, flag_cap,
                                   reinterpret_cast<unsigned long long*>(ix.keys)));
  return cudaGetLastError();
}

size_t proj_hash_tc_smem(int Wp, bool lo) { return tc_smem_bytes(Wp, lo); }

}  // namespace momenti
