// The passes over binary features on the FP8 tensor cores (tcgen05.mma
// kind::f8f6f4, E4M3 x E4M3 -> FP32): the sketch U = X Omega (Eq. 1) and pass
// F = U^T X (Algorithm 2 step 2, Algorithm 4's F += U_s^T X_s) for FP8 E4M3 X
// with the very sparse Omega.
//
// Number formats.  Omega's entries 0 and +-1 are exact in E4M3, and so are
// the 0/1 features of the paper's binary data, so the sketch's products are
// exact; every sum of E4M3 values below 2^15 in magnitude is a multiple of
// 2^-9 below 2^24 ulps and therefore exact in FP32 whatever the rounding of the
// accumulation, so U comes out exact.  Pass F takes U as E4M3 bytes: exact
// whenever every entry of U is representable (integers up to 16 always are;
// the sketch checks every entry and raises a flag otherwise, and the BF16
// pass F then runs instead).  For binary X the products U x are then integers
// and the FP32 sums of one row chunk stay below 2^24 (chunks of at most 2^20
// rows, |U| <= 16), so F is exact too.
//
// Sketch, f8_sketch_kernel (persistent, one CTA per SM): D = X_tile Omega
// with M = 128 rows of X, N = k padded to 32, K = n in steps of 128 bytes.  A
// (the X tile) and B (Omega^T, built once in E4M3, k x n) are both K-major and
// arrive by TMA in 128-byte-swizzled boxes.  Two TMEM accumulators alternate,
// so the epilogue (four warps, one TMEM lane quarter each) writes U for one
// tile while the tensor core accumulates the next.
//
// Pass F, f8_chain_kernel (one unit per CTA): D = U^T X over one chunk of rows
// for a 256-column tile of X, both halves of k at once (two 128-row M halves,
// 2 x 256 TMEM columns).  Both operands are MN-major (the reduction runs over
// the rows of two row-major sources): boxes of 128 rows x 128 bytes, the
// swizzle atoms 8 rows x 128 bytes.  The chunks of one tile are read by 16
// CTAs at about the same time, so U is read from HBM about once.  Each CTA
// writes one FP32 partial of F; the partials are summed in fixed order.
//
// Roles: warps 0-3 epilogue, warp 4 allocates TMEM and issues the MMAs (one
// thread), warp 5 the TMA copies (one thread).  Every wait is bounded (2 s of
// %globaltimer): on expiry the kernel records ST_TIMEOUT, the roles stop, the
// producer waits (bounded) for its copies in flight, the MMA thread for its
// products, and TMEM is freed.
#include "common.cuh"
#include "kernels.h"
#include "philox.cuh"
#include "tc_ptx.cuh"
#include "tma.h"

namespace lspca {
namespace f8 {

constexpr uint64_t kWaitNs = 2000000000ull;
constexpr uint64_t kDrainNs = 100000000ull;
constexpr int kThreads = 192;
constexpr int kEpiWarps = 4, kMmaWarp = 4, kProdWarp = 5;
constexpr int kBK = 128;                 // K per stage: 128 bytes (sketch) or 128 rows (pass F)
constexpr uint32_t kBox = kBK * 128;     // one 128 x 128-byte box: 16 KB

// kind::f8f6f4 instruction descriptor: FP32 accumulator, A and B E4M3 (format
// 0), majorness (1 = MN-major), N and M.
__host__ __device__ constexpr uint32_t idesc_f8(int M, int N, int a_mn, int b_mn) {
  return (1u << 4) | ((uint32_t)a_mn << 15) | ((uint32_t)b_mn << 16) | ((uint32_t)(N >> 3) << 17) |
         ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_f8(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                       uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}

// Bounded wait; on expiry the status and the CTA's abort flag are set.
__device__ __forceinline__ bool wait_or_abort(uint64_t* bar, uint32_t parity, volatile int* abort, int* status) {
  if (*abort) return false;
  if (ptx::mbar_wait(bar, parity, kWaitNs)) return true;
  *abort = 1;
  atomicOr(status, ST_TIMEOUT);
  return false;
}

// E4M3 byte of an FP32 value (round to nearest even, saturating).
__device__ __forceinline__ uint8_t to_e4m3(float v) {
  return (uint8_t)__nv_cvt_float_to_fp8(v, __NV_SATFINITE, __NV_E4M3);
}
__device__ __forceinline__ float from_e4m3(uint8_t b) {
  __nv_fp8_e4m3 t;
  t.__x = b;
  return (float)t;
}

// ---------------------------------------------------------------------------
// Omega^T in E4M3 (np x n, row pitch ldo bytes; rows k .. np-1 zero): 0x00,
// 0x38 (+1), 0xB8 (-1).
__global__ void omega_t_e4m3_kernel(lspca_omega om, int64_t n, int64_t ldo, int k, int np, uint8_t* out) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int nb = np / 4;
  if (idx >= n * nb) return;
  const int64_t j = idx / nb;
  const int b = (int)(idx % nb);
  uint4 w = make_uint4(0u, 0u, 0u, 0u);
  if (4 * b < k) w = omega_words(om.seed, (uint32_t)j, (uint32_t)b, kTagSparse);
  const uint64_t t = sparse_threshold(om.p);
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int l = 4 * b + q;
    const uint64_t r = word_of(w, q);
    uint8_t v = 0;
    if (l < k && r < 2 * t) v = r < t ? 0xB8 : 0x38;
    out[(int64_t)l * ldo + j] = v;
  }
}

// ---------------------------------------------------------------------------
struct SketchParams {
  int64_t m, n;
  int k, np;          // np = k padded to 32 (N of the MMA)
  int64_t tiles;      // 128-row tiles of X
  float* U;           // m x k FP32 (nullable)
  uint8_t* U8;        // m x np E4M3
  float* umax;
  int* inexact;       // set when some U is not exactly an E4M3 value
  int* status;
  const int* run_if;  // nullable: the kernel does nothing unless *run_if != 0
};

template <int NP>
struct SkCfg {
  static constexpr uint32_t A_BYTES = kBox;             // 128 rows x 128 bytes
  static constexpr uint32_t B_BYTES = NP * 128;         // NP rows x 128 bytes
  static constexpr uint32_t STAGE = A_BYTES + B_BYTES;
  static constexpr int STAGES = STAGE * 4 <= 200 * 1024 ? 4 : 3;
  static constexpr size_t SMEM = 1024 + (size_t)STAGES * STAGE + 512;
  static constexpr uint32_t TMEM_COLS = 2 * NP <= 128 ? 128 : (2 * NP <= 256 ? 256 : 512);
};

template <int NP>
__global__ void __launch_bounds__(kThreads, 1) f8_sketch_kernel(const __grid_constant__ CUtensorMap tmx,
                                                                const __grid_constant__ CUtensorMap tmo,
                                                                SketchParams p) {
  using C = SkCfg<NP>;
  if (p.run_if && *p.run_if == 0) return;  // uniform: the gated second run is not needed
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint64_t* bars = (uint64_t*)(smem + (size_t)C::STAGES * C::STAGE);
  uint64_t* full = bars;
  uint64_t* empty = full + C::STAGES;
  uint64_t* tfull = empty + C::STAGES;
  uint64_t* tempty = tfull + 2;
  uint64_t* drain = tempty + 2;
  uint32_t* tslot = (uint32_t*)(drain + 1);
  volatile int* abort = (volatile int*)(tslot + 1);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t ksteps = (p.n + kBK - 1) / kBK;
  if (threadIdx.x == 0) {
    for (int s = 0; s < C::STAGES; ++s) {
      ptx::mbar_init(&full[s], 1);
      ptx::mbar_init(&empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      ptx::mbar_init(&tfull[b], 1);
      ptx::mbar_init(&tempty[b], kEpiWarps);
    }
    ptx::mbar_init(drain, 1);
    *abort = 0;
    ptx::fence_mbar_init();
  }
  if (warp == kMmaWarp) ptx::tmem_alloc(tslot, C::TMEM_COLS);
  ptx::tc_fence_before();
  __syncthreads();
  ptx::tc_fence_after();
  const uint32_t tmem = *tslot;

  if (warp == kProdWarp) {
    if (lane == 0) {
      int64_t it = 0;
      for (int64_t t = blockIdx.x; t < p.tiles && !*abort; t += gridDim.x) {
        for (int64_t ks = 0; ks < ksteps; ++ks, ++it) {
          const int slot = (int)(it % C::STAGES);
          const uint32_t par = (uint32_t)((it / C::STAGES) & 1) ^ 1u;
          if (!wait_or_abort(&empty[slot], par, abort, p.status)) break;
          uint8_t* st = smem + (size_t)slot * C::STAGE;
          ptx::mbar_arrive_expect_tx(&full[slot], C::STAGE);
          ptx::tma_load_2d(ptx::smem_u32(st), &tmx, (int)(ks * kBK), (int)(t * 128), &full[slot]);
          ptx::tma_load_2d(ptx::smem_u32(st + C::A_BYTES), &tmo, (int)(ks * kBK), 0, &full[slot]);
        }
      }
      if (*abort) {  // copies in flight land before the CTA leaves
        for (int64_t q = it - C::STAGES; q < it; ++q) {
          if (q < 0) continue;
          ptx::mbar_wait(&full[q % C::STAGES], (uint32_t)((q / C::STAGES) & 1), kDrainNs);
        }
      }
    }
  } else if (warp == kMmaWarp) {
    if (lane == 0) {
      constexpr uint32_t idesc = idesc_f8(128, NP, 0, 0);
      int64_t it = 0, lt = 0;
      for (int64_t t = blockIdx.x; t < p.tiles && !*abort; t += gridDim.x, ++lt) {
        const int b = (int)(lt & 1);
        if (!wait_or_abort(&tempty[b], (uint32_t)((lt >> 1) & 1) ^ 1u, abort, p.status)) break;
        ptx::tc_fence_after();
        const uint32_t d = tmem + (uint32_t)(b * NP);
        for (int64_t ks = 0; ks < ksteps; ++ks, ++it) {
          const int slot = (int)(it % C::STAGES);
          if (!wait_or_abort(&full[slot], (uint32_t)((it / C::STAGES) & 1), abort, p.status)) break;
          ptx::tc_fence_after();
          const uint32_t sa = ptx::smem_u32(smem + (size_t)slot * C::STAGE);
          const uint64_t ad = ptx::desc_sw128(sa, 16, 1024);
          const uint64_t bd = ptx::desc_sw128(sa + C::A_BYTES, 16, 1024);
#pragma unroll
          for (int kk = 0; kk < 4; ++kk)
            mma_f8(d, ptx::desc_advance(ad, kk * 32), ptx::desc_advance(bd, kk * 32), idesc,
                   (ks > 0 || kk > 0) ? 1u : 0u);
          ptx::mma_commit(&empty[slot]);
        }
        if (*abort) break;
        ptx::mma_commit(&tfull[b]);
      }
      ptx::mma_commit(drain);  // all products of this thread done before TMEM is freed
      ptx::mbar_wait(drain, 0, kDrainNs);
    }
  } else {
    // epilogue: warp w reads TMEM lanes 32w .. 32w + 31 (rows of the tile)
    int64_t lt = 0;
    float mx = 0.f;
    bool inexact = false;
    for (int64_t t = blockIdx.x; t < p.tiles; t += gridDim.x, ++lt) {
      const int b = (int)(lt & 1);
      if (!wait_or_abort(&tfull[b], (uint32_t)((lt >> 1) & 1), abort, p.status)) break;
      ptx::tc_fence_after();
      const int64_t row = t * 128 + warp * 32 + lane;
      const bool live = row < p.m;
#pragma unroll 1
      for (int c0 = 0; c0 < NP; c0 += 32) {
        uint32_t r[32];
        ptx::tmem_ld32(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(b * NP + c0), r);
        if (live) {
          uint32_t pk[8];
#pragma unroll
          for (int q = 0; q < 8; ++q) {
            uint32_t word = 0;
#pragma unroll
            for (int e = 0; e < 4; ++e) {
              const int c = c0 + 4 * q + e;
              const float v = c < p.k ? __uint_as_float(r[4 * q + e]) : 0.f;
              const uint8_t e8 = to_e4m3(v);
              inexact |= from_e4m3(e8) != v;
              mx = fmaxf(mx, fabsf(v));
              word |= (uint32_t)e8 << (8 * e);
            }
            pk[q] = word;
          }
          uint4* dst8 = reinterpret_cast<uint4*>(p.U8 + row * p.np + c0);
          dst8[0] = make_uint4(pk[0], pk[1], pk[2], pk[3]);
          dst8[1] = make_uint4(pk[4], pk[5], pk[6], pk[7]);
          if (p.U) {
            float* ur = p.U + row * p.k;
            if (c0 + 32 <= p.k && (p.k & 3) == 0) {
#pragma unroll
              for (int q = 0; q < 8; ++q)
                reinterpret_cast<float4*>(ur + c0)[q] =
                    make_float4(__uint_as_float(r[4 * q]), __uint_as_float(r[4 * q + 1]),
                                __uint_as_float(r[4 * q + 2]), __uint_as_float(r[4 * q + 3]));
            } else {
              for (int e = 0; e < 32 && c0 + e < p.k; ++e) ur[c0 + e] = __uint_as_float(r[e]);
            }
          }
        }
      }
      ptx::tc_fence_before();
      __syncwarp();
      if (lane == 0) ptx::mbar_arrive(&tempty[b]);
    }
    mx = warp_max(mx);
    if (lane == 0 && mx > 0.f) atomic_max_nonneg(p.umax, mx);
    if (__any_sync(0xffffffffu, inexact) && lane == 0) atomicOr(p.inexact, 1);
  }
  ptx::tc_fence_before();
  __syncthreads();
  if (warp == kMmaWarp) {
    ptx::tc_fence_after();
    ptx::tmem_dealloc(tmem, C::TMEM_COLS);
  }
}

// ---------------------------------------------------------------------------
struct ChainParams {
  int64_t m, n;
  int k, mh;          // mh: 128-row halves of k (1 or 2)
  int tiles, chunks;  // 256-column tiles of X, row chunks
  int64_t rows;       // rows per chunk (a multiple of 128)
  float* part;        // chunks x k x n FP32
  const int* inexact; // set: U is not exact in E4M3, this pass does nothing
  int* status;
};

constexpr uint32_t kChA = kBox;        // one M half of U^T: 128 rows x 128 bytes
constexpr uint32_t kChB = 2 * kBox;    // X: two boxes of 128 rows x 128 bytes (N = 256)
constexpr uint32_t kChStage = 2 * kChA + kChB;
constexpr int kChStages = 3;
constexpr size_t kChSmem = 1024 + (size_t)kChStages * kChStage + 512;

__global__ void __launch_bounds__(kThreads, 1) f8_chain_kernel(const __grid_constant__ CUtensorMap tmu,
                                                               const __grid_constant__ CUtensorMap tmx,
                                                               ChainParams p) {
  if (*p.inexact) return;  // uniform: the BF16 pass F runs instead
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint64_t* bars = (uint64_t*)(smem + (size_t)kChStages * kChStage);
  uint64_t* full = bars;
  uint64_t* empty = full + kChStages;
  uint64_t* done = empty + kChStages;
  uint64_t* drain = done + 1;
  uint32_t* tslot = (uint32_t*)(drain + 1);
  volatile int* abort = (volatile int*)(tslot + 1);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int tile = (int)(blockIdx.x % p.tiles), chunk = (int)(blockIdx.x / p.tiles);
  const int64_t r0 = (int64_t)chunk * p.rows;
  const int64_t r1 = min(p.m, r0 + p.rows);
  const int64_t steps = (r1 - r0 + kBK - 1) / kBK;
  if (threadIdx.x == 0) {
    for (int s = 0; s < kChStages; ++s) {
      ptx::mbar_init(&full[s], 1);
      ptx::mbar_init(&empty[s], 1);
    }
    ptx::mbar_init(done, 1);
    ptx::mbar_init(drain, 1);
    *abort = 0;
    ptx::fence_mbar_init();
  }
  if (warp == kMmaWarp) ptx::tmem_alloc(tslot, 512);
  ptx::tc_fence_before();
  __syncthreads();
  ptx::tc_fence_after();
  const uint32_t tmem = *tslot;

  if (warp == kProdWarp) {
    if (lane == 0) {
      int64_t s = 0;
      for (; s < steps; ++s) {
        const int slot = (int)(s % kChStages);
        if (!wait_or_abort(&empty[slot], (uint32_t)((s / kChStages) & 1) ^ 1u, abort, p.status)) break;
        uint8_t* st = smem + (size_t)slot * kChStage;
        const int y = (int)(r0 + s * kBK);
        ptx::mbar_arrive_expect_tx(&full[slot], (uint32_t)p.mh * kChA + kChB);
        for (int h = 0; h < p.mh; ++h) ptx::tma_load_2d(ptx::smem_u32(st + h * kChA), &tmu, h * 128, y, &full[slot]);
        ptx::tma_load_2d(ptx::smem_u32(st + 2 * kChA), &tmx, tile * 256, y, &full[slot]);
        ptx::tma_load_2d(ptx::smem_u32(st + 2 * kChA + kBox), &tmx, tile * 256 + 128, y, &full[slot]);
      }
      if (*abort) {
        for (int64_t q = s - kChStages; q < s; ++q) {
          if (q < 0) continue;
          ptx::mbar_wait(&full[q % kChStages], (uint32_t)((q / kChStages) & 1), kDrainNs);
        }
      }
    }
  } else if (warp == kMmaWarp) {
    if (lane == 0) {
      constexpr uint32_t idesc = idesc_f8(128, 256, 1, 1);
      for (int64_t s = 0; s < steps; ++s) {
        const int slot = (int)(s % kChStages);
        if (!wait_or_abort(&full[slot], (uint32_t)((s / kChStages) & 1), abort, p.status)) break;
        ptx::tc_fence_after();
        const uint32_t sa = ptx::smem_u32(smem + (size_t)slot * kChStage);
        const uint64_t bd = ptx::desc_sw128(sa + 2 * kChA, kBox, 1024);
        for (int h = 0; h < p.mh; ++h) {
          const uint64_t ad = ptx::desc_sw128(sa + h * kChA, kBox, 1024);
#pragma unroll
          for (int kk = 0; kk < 4; ++kk)
            mma_f8(tmem + (uint32_t)(h * 256), ptx::desc_advance(ad, kk * 4096), ptx::desc_advance(bd, kk * 4096),
                   idesc, (s > 0 || kk > 0) ? 1u : 0u);
        }
        ptx::mma_commit(&empty[slot]);
      }
      ptx::mma_commit(done);
      if (*abort) ptx::mbar_wait(done, 0, kDrainNs);
    }
  } else {
    // epilogue: row l = 128 h + 32 w + lane of F, 256 columns of the tile
    if (wait_or_abort(done, 0, abort, p.status)) {
      ptx::tc_fence_after();
      float* part = p.part + (int64_t)chunk * p.k * p.n;
      const int64_t j0 = (int64_t)tile * 256;
      for (int h = 0; h < p.mh; ++h) {
        const int l = h * 128 + warp * 32 + lane;
#pragma unroll 1
        for (int c0 = 0; c0 < 256; c0 += 32) {
          uint32_t r[32];
          ptx::tmem_ld32(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(h * 256 + c0), r);
          if (l >= p.k) continue;
          float* dst = part + (int64_t)l * p.n + j0 + c0;
          if (j0 + c0 + 32 <= p.n && (p.n & 3) == 0) {
#pragma unroll
            for (int q = 0; q < 8; ++q)
              reinterpret_cast<float4*>(dst)[q] =
                  make_float4(__uint_as_float(r[4 * q]), __uint_as_float(r[4 * q + 1]),
                              __uint_as_float(r[4 * q + 2]), __uint_as_float(r[4 * q + 3]));
          } else {
            for (int e = 0; e < 32 && j0 + c0 + e < p.n; ++e) dst[e] = __uint_as_float(r[e]);
          }
        }
      }
    }
  }
  ptx::tc_fence_before();
  __syncthreads();
  if (warp == kMmaWarp) {
    ptx::tc_fence_after();
    ptx::tmem_dealloc(tmem, 512);
  }
}

// U (FP32, m x k) -> E4M3 bytes (m x np), with the flag raised when some
// entry is not exactly an E4M3 value (pass F of a caller-supplied U).
__global__ void u_to_e4m3_kernel(const float* __restrict__ U, int64_t m, int k, int np, uint8_t* __restrict__ U8,
                                 int* inexact) {
  bool bad = false;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < m * np; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = e / np;
    const int c = (int)(e - r * np);
    const float v = c < k ? U[r * k + c] : 0.f;
    const uint8_t b = to_e4m3(v);
    bad |= from_e4m3(b) != v;
    U8[e] = b;
  }
  if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicOr(inexact, 1);
}

// Sum of the chunk partials (compensated FP32, fixed order) into F, gated:
// runs only when U was exact in E4M3.
__global__ void f8_reduce_kernel(const float* __restrict__ part, int chunks, int64_t count, double* __restrict__ F,
                                 const int* inexact) {
  if (*inexact) return;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < count; e += (int64_t)gridDim.x * blockDim.x) {
    float s = 0.f, c = 0.f;
    for (int q = 0; q < chunks; ++q) {
      const float x = part[(int64_t)q * count + e];
      const float t = s + x;
      const float bp = t - s;
      c += (s - (t - bp)) + (x - bp);
      s = t;
    }
    F[e] = (double)s + (double)c;
  }
}

}  // namespace f8

int f8_np(int k) { return (k + 31) / 32 * 32; }

static int64_t pitch16b(int64_t n) { return (n + 15) / 16 * 16; }

size_t f8_ws_bytes(int64_t m, int64_t n, int k, int num_sms) {
  const int np = f8_np(k);
  const int tiles = (int)((n + 255) / 256);
  int chunks = tiles >= num_sms ? 1 : num_sms / tiles;
  int64_t rows = ((m + chunks - 1) / chunks + 127) / 128 * 128;
  if (rows > (1 << 20)) rows = 1 << 20;  // exact integer sums for |U| <= 16, binary X
  chunks = (int)((m + rows - 1) / rows);
  auto al = [](size_t b) { return (b + 255) / 256 * 256; };
  return al((size_t)np * pitch16b(n)) + al((size_t)m * np) + al((size_t)chunks * k * n * 4) + 256;
}

namespace {
struct F8Ws {
  uint8_t* omt;
  uint8_t* U8;
  float* part;
  int* inexact;
  int chunks;
  int64_t rows;
  int tiles;
};
F8Ws carve_f8(void* ws, int64_t m, int64_t n, int k, int num_sms) {
  F8Ws w;
  const int np = f8_np(k);
  w.tiles = (int)((n + 255) / 256);
  int chunks = w.tiles >= num_sms ? 1 : num_sms / w.tiles;
  int64_t rows = ((m + chunks - 1) / chunks + 127) / 128 * 128;
  if (rows > (1 << 20)) rows = 1 << 20;
  w.rows = rows;
  w.chunks = (int)((m + rows - 1) / rows);
  auto al = [](size_t b) { return (b + 255) / 256 * 256; };
  char* p = (char*)ws;
  w.omt = (uint8_t*)p;
  p += al((size_t)np * pitch16b(n));
  w.U8 = (uint8_t*)p;
  p += al((size_t)m * np);
  w.part = (float*)p;
  p += al((size_t)w.chunks * k * n * 4);
  w.inexact = (int*)p;
  return w;
}
}  // namespace

int* f8_inexact_flag(void* ws, int64_t m, int64_t n, int k, int num_sms) {
  return carve_f8(ws, m, n, k, num_sms).inexact;
}

bool launch_f8_sketch(Launcher& L, const void* X, int64_t m, int64_t n, int64_t ldx, int k, const lspca_omega& om,
                      void* ws, float* U, float* umax, int* status, bool again) {
  F8Ws w = carve_f8(ws, m, n, k, L.num_sms);
  const int np = f8_np(k);
  if (!again) {
    cudaMemsetAsync(w.inexact, 0, sizeof(int), L.stream);
    const int64_t total = n * (np / 4);
    f8::omega_t_e4m3_kernel<<<(unsigned)((total + 255) / 256), 256, 0, L.stream>>>(om, n, pitch16b(n), k, np,
                                                                                    w.omt);
  }
  CUtensorMap tmx, tmo;
  if (!make_tmap_2d_sw128(&tmx, X, CU_TENSOR_MAP_DATA_TYPE_UINT8, 1, (uint64_t)m, (uint64_t)n, (uint64_t)ldx, 128,
                          128) ||
      !make_tmap_2d_sw128(&tmo, w.omt, CU_TENSOR_MAP_DATA_TYPE_UINT8, 1, (uint64_t)np, (uint64_t)n,
                          (uint64_t)pitch16b(n), (uint32_t)np, 128))
    return false;
  f8::SketchParams p{m, n, k, np, (m + 127) / 128, U, w.U8, umax, w.inexact, status, again ? w.inexact : nullptr};
  const int64_t grid = p.tiles < L.num_sms ? p.tiles : L.num_sms;
  auto go = [&](auto kern, size_t smem) {
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    kern<<<(unsigned)grid, f8::kThreads, smem, L.stream>>>(tmx, tmo, p);
  };
  switch (np) {
    case 32: go(f8::f8_sketch_kernel<32>, f8::SkCfg<32>::SMEM); break;
    case 64: go(f8::f8_sketch_kernel<64>, f8::SkCfg<64>::SMEM); break;
    case 96: go(f8::f8_sketch_kernel<96>, f8::SkCfg<96>::SMEM); break;
    case 128: go(f8::f8_sketch_kernel<128>, f8::SkCfg<128>::SMEM); break;
    case 160: go(f8::f8_sketch_kernel<160>, f8::SkCfg<160>::SMEM); break;
    case 192: go(f8::f8_sketch_kernel<192>, f8::SkCfg<192>::SMEM); break;
    case 224: go(f8::f8_sketch_kernel<224>, f8::SkCfg<224>::SMEM); break;
    default: go(f8::f8_sketch_kernel<256>, f8::SkCfg<256>::SMEM); break;
  }
  L.count(2);
  return true;
}

void launch_f8_u8(Launcher& L, const float* U, int64_t m, int k, void* ws, int64_t n) {
  F8Ws w = carve_f8(ws, m, n, k, L.num_sms);
  const int np = f8_np(k);
  cudaMemsetAsync(w.inexact, 0, sizeof(int), L.stream);
  int64_t blocks = (m * np + 255) / 256;
  if (blocks > 8 * L.num_sms) blocks = 8 * L.num_sms;
  f8::u_to_e4m3_kernel<<<(unsigned)blocks, 256, 0, L.stream>>>(U, m, k, np, w.U8, w.inexact);
  L.count(1);
}

bool launch_f8_chain(Launcher& L, const void* X, int64_t m, int64_t n, int64_t ldx, int k, void* ws, double* F,
                     int* status) {
  F8Ws w = carve_f8(ws, m, n, k, L.num_sms);
  const int np = f8_np(k);
  CUtensorMap tmu, tmx;
  if (!make_tmap_2d_sw128(&tmu, w.U8, CU_TENSOR_MAP_DATA_TYPE_UINT8, 1, (uint64_t)m, (uint64_t)np, (uint64_t)np, 128,
                          128) ||
      !make_tmap_2d_sw128(&tmx, X, CU_TENSOR_MAP_DATA_TYPE_UINT8, 1, (uint64_t)m, (uint64_t)n, (uint64_t)ldx, 128,
                          128))
    return false;
  f8::ChainParams p{m, n, k, k > 128 ? 2 : 1, w.tiles, w.chunks, w.rows, w.part, w.inexact, status};
  cudaFuncSetAttribute(f8::f8_chain_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)f8::kChSmem);
  f8::f8_chain_kernel<<<(unsigned)(w.tiles * w.chunks), f8::kThreads, f8::kChSmem, L.stream>>>(tmu, tmx, p);
  const int64_t cnt = (int64_t)k * n;
  int blocks = (int)((cnt + 255) / 256);
  if (blocks > 8 * L.num_sms) blocks = 8 * L.num_sms;
  f8::f8_reduce_kernel<<<blocks, 256, 0, L.stream>>>(w.part, w.chunks, cnt, F, w.inexact);
  L.count(2);
  return true;
}

}  // namespace lspca
