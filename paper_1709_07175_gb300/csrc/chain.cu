// Pass F on sm_103a tensor cores with TMA-fed operands: F = U^T X
// (Algorithm 4's F += U_s^T X_s, Algorithm 2 step 2) and, optionally, the
// Gram G = U^T U (Lemma 1 / Prop. 1).
//
// D[c, j] = sum over the rows i of one m-chunk of U[i, c] B[i, j], B = X (or U
// for the Gram): a GEMM whose reduction runs over the rows of two row-major
// sources, so both operands are MN-major.  M = k (one or two 128-row halves),
// N = a 256-column (128 when k > 128) tile of B, K = rows.
//
// Number formats (the same as the tensor-core reduction map):
//  * FP32 X: U and X are split into FP16 pairs v s = hi + lo with power-of-two
//    scales s from max|U| and max|X| (|v s| <= 2^14); three products
//    hi*hi + hi*lo + lo*hi carry ~22 significant bits.
//  * BF16 X: X is exact, U is split into a BF16 pair (no scale), two products.
//  * E4M3 X: widened exactly to BF16, U as a BF16 pair, two products.
//  * Gram: B = U, both FP16 pairs with the max|U| scale, three products.
//
// U is split once per fit by split_u_kernel into two row-major 16-bit arrays
// (pitch ku = k rounded up to 8), so every CTA loads the A operand with tiled
// TMA copies (boxes of BK rows x 64 columns, 128-byte swizzle: exactly the
// MN-major SW128 operand layout; rows past m and columns past k arrive as
// zeros).  For BF16 X and for the Gram the B operand is loaded the same way
// and the kernel has no converter warps; FP32 and E4M3 X are converted by
// converter warps that load X rows with 16-byte global loads one step ahead
// (two register buffers in ping-pong).  (L2 prefetches of the rows a few steps
// ahead were measured on GB300 to slow this pass down: bulk prefetches by a
// third, per-thread line prefetches two steps ahead by 6 %.)
//
// Accumulation.  Measured on GB300, the FP32 accumulation of tcgen05.mma into
// TMEM behaves like round-toward-zero (its error is biased and grows with the
// number of accumulating instructions), so the tensor core accumulates only
// segments of SEG k-steps (SEG * BK rows) into a TMEM accumulator A; the
// epilogue warps fold each finished segment into a round-to-nearest FP32
// running sum S in TMEM and write S, scaled back, as the unit's FP32 partial
// after its last segment.  Eight epilogue warps fold in parallel, since each
// fold is a chain of TMEM load / store round trips.  Partials of the m-chunks
// are summed in FP64 in fixed order (tc_chain_reduce).
//
// Kernel structure (one persistent CTA per SM; a unit = (m-chunk, N tile)):
//   warps 0..CW-1      converters (16 for FP32 X, 8 for E4M3 X, none otherwise);
//   warps CW..CW+7     epilogue (two per TMEM lane quarter, half the columns each);
//   warp  CW+8         TMEM allocation, the thread that issues tcgen05.mma;
//   warp  CW+9         producer: TMA copies of each stage (lane 0).
// Ring of STAGES shared-memory stages; per stage the mbarriers tfull (TMA
// bytes), full (converter warps), empty (tcgen05.commit).  Every wait is
// bounded (2 s of %globaltimer): on expiry the kernel records ST_TIMEOUT,
// stops issuing work, waits (bounded) for its copies and MMAs in flight and
// frees TMEM.
#include "common.cuh"
#include "tc.h"
#include "tc_ptx.cuh"
#include "tma.h"

namespace lspca {
namespace pf {

constexpr int BK = 32;       // rows (K) per stage
constexpr uint64_t kWaitNs = 2000000000ull;
constexpr uint64_t kDrainNs = 100000000ull;

enum Mode { M_F32 = 0, M_BF16 = 1, M_E4M3 = 2, M_GRAM = 3 };
constexpr int kConvBuffers = 2;

template <int MODE, int MH, int NACC>
struct Cfg {
  static_assert(NACC == 1 || (NACC == 2 && MH == 1), "double-buffered A with one M half only");
  // The Gram with k <= 128: B = U is the A tile itself (the same rows, the
  // same MN-major layout), so it is loaded once and read as both operands
  static constexpr bool SHARE_B = MODE == M_GRAM && MH == 1;
  static constexpr int BN = (SHARE_B || MH == 2 || NACC == 2) ? 128 : 256;
  static constexpr int WA = 128 * MH;
  static constexpr bool CONV = (MODE == M_F32 || MODE == M_E4M3);
  static constexpr bool F16 = (MODE == M_F32 || MODE == M_GRAM);  // FP16 pairs, else BF16
  static constexpr int NB = F16 ? 2 : 1;                          // B operand parts
  static constexpr int CW = MODE == M_F32 ? 16 : (CONV ? 8 : 0);
  static constexpr int CT = CW * 32;
  static constexpr int EW_N = 8;  // epilogue warps: two per TMEM lane quarter, each folds half the columns
  static constexpr int EPI0 = CW;  // a multiple of 4, so warp EPI0 + e owns TMEM lane quarter e % 4
  static constexpr int MMA_W = CW + EW_N;
  static constexpr int PROD_W = CW + EW_N + 1;
  static constexpr int THREADS = (CW + EW_N + 2) * 32;
  static constexpr uint32_t BOX = BK * 128;        // one TMA box: BK rows x 64 16-bit columns
  static constexpr uint32_t A_BYTES = BK * WA * 2;  // one part of A
  static constexpr uint32_t B_BYTES = BK * BN * 2;  // one part of B
  static constexpr uint32_t STAGE_BYTES = 2 * A_BYTES + (SHARE_B ? 0u : NB * B_BYTES);
  static constexpr int STAGES = STAGE_BYTES <= 24576 ? 8 : STAGE_BYTES <= 32768 ? 6 : 4;
  static constexpr uint32_t TX = 2 * A_BYTES + ((CONV || SHARE_B) ? 0u : NB * B_BYTES);
  static constexpr uint32_t SBO_B = (BN / 64) * 1024;  // converter layout of B: K atom groups
  static constexpr int ELEM = (MODE == M_F32) ? 4 : 1;  // converter modes: bytes per X element
  static constexpr int B_VEC = CONV ? BK * BN * ELEM / 16 / CT : 1;  // 16-byte loads per thread per step
  // k-steps the tensor core accumulates per segment: 8 for F (measured mean
  // relative bias of F on GB300: -8e-7, nearly uniform across entries), 4 for
  // the Gram, whose entries are all compared to one norm (-4e-7)
  static constexpr int SEG = MODE == M_GRAM ? 4 : 8;
  static constexpr int NBUF = kConvBuffers;  // register buffers of the converters (loads NBUF - 1 steps ahead)
  static constexpr size_t SMEM = 1024 + (size_t)STAGES * STAGE_BYTES + 256 + 8192;
  // TMEM: NACC segment accumulators of MH x BN columns, then the running sum S
  static constexpr uint32_t ACC_COLS = MH * BN;
  static constexpr uint32_t S_COL = NACC * ACC_COLS;
  static constexpr uint32_t TMEM_COLS = 512;
  static_assert(S_COL + ACC_COLS <= TMEM_COLS, "TMEM budget");
};

struct Params {
  const void* X;  // B source of the converter modes (row-major, ld ldb)
  int64_t ldb;
  int64_t nb;     // columns of the B source
  int64_t m;
  int k;
  int tiles;      // N tiles of the B source
  int chunks;     // m-chunks; chunk c takes the BK-row blocks c, c + chunks, c + 2 chunks, ...
  int64_t nblocks;  // BK-row blocks of m
  float* part;    // chunks x k x nb FP32 partials
  const float* amax_b;  // max|B source| (FP32 X and Gram scales)
  const float* amax_u;  // max|U|
  int* status;
  const int* gate;      // nullable: the pass runs only when *gate != 0
};

// Power-of-two scale s with |v s| < 2^14 for |v| <= amax (1 for amax 0 / non-finite).
__device__ __forceinline__ float pow2_scale(float amax) {
  if (!(amax > 0.f) || !isfinite(amax)) return 1.f;
  int e;
  frexpf(amax, &e);  // amax < 2^e
  return ldexpf(1.f, 14 - e);
}

__device__ __forceinline__ uint32_t pack_h2(float a, float b) {
  __half2 h = __floats2half2_rn(a, b);
  return *reinterpret_cast<uint32_t*>(&h);
}
__device__ __forceinline__ uint32_t pack_b2(float a, float b) {
  __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
  return *reinterpret_cast<uint32_t*>(&h);
}

// (a, b) -> hi pair and lo pair, FP16: hi = fp16(v), lo = fp16(v - hi).
__device__ __forceinline__ void split_h2(float a, float b, uint32_t& hi, uint32_t& lo) {
  __half2 h = __floats2half2_rn(a, b);
  const float2 f = __half22float2(h);
  hi = *reinterpret_cast<uint32_t*>(&h);
  lo = pack_h2(a - f.x, b - f.y);
}
__device__ __forceinline__ void split_b2(float a, float b, uint32_t& hi, uint32_t& lo) {
  __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
  const float2 f = __bfloat1622float2(h);
  hi = *reinterpret_cast<uint32_t*>(&h);
  lo = pack_b2(a - f.x, b - f.y);
}

__device__ __forceinline__ void sts64(uint32_t addr, uint32_t x, uint32_t y) {
  asm volatile("st.shared.v2.b32 [%0], {%1, %2};" ::"r"(addr), "r"(x), "r"(y) : "memory");
}
__device__ __forceinline__ void sts128(uint32_t addr, uint4 v) {
  asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(addr), "r"(v.x), "r"(v.y), "r"(v.z), "r"(v.w)
               : "memory");
}
__device__ __forceinline__ uint4 ldg16(const void* p) {
  uint4 v;
  asm volatile("ld.global.nc.L1::no_allocate.v4.u32 {%0, %1, %2, %3}, [%4];"
               : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
               : "l"(p));
  return v;
}

// U (m x k FP32, ld k, k % 4 == 0) -> hi, lo (m x ku 16-bit): FP16 pairs of
// U s (s = pow2_scale(max|U|)) or BF16 pairs of U.
template <bool F16>
__global__ void split_u_kernel(const float* __restrict__ U, int64_t m, int k, int64_t ku,
                               const float* __restrict__ amax, uint16_t* __restrict__ hi, uint16_t* __restrict__ lo,
                               const int* gate) {
  if (gate && *gate == 0) return;
  const float s = F16 ? pow2_scale(*amax) : 1.f;
  const int k4 = k / 4;
  const int64_t total = m * k4;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = e / k4;
    const int c = (int)(e - r * k4) * 4;
    const float4 v = __ldg(reinterpret_cast<const float4*>(U + r * k + c));
    uint32_t h0, l0, h1, l1;
    if (F16) {
      split_h2(v.x * s, v.y * s, h0, l0);
      split_h2(v.z * s, v.w * s, h1, l1);
    } else {
      split_b2(v.x, v.y, h0, l0);
      split_b2(v.z, v.w, h1, l1);
    }
    *reinterpret_cast<uint2*>(hi + r * ku + c) = make_uint2(h0, h1);
    *reinterpret_cast<uint2*>(lo + r * ku + c) = make_uint2(l0, l1);
  }
}

template <int MODE, int MH, int NACC>
__global__ void __launch_bounds__(Cfg<MODE, MH, NACC>::THREADS, 1)
    passf_kernel(const __grid_constant__ CUtensorMap tm_ahi, const __grid_constant__ CUtensorMap tm_alo,
                 const __grid_constant__ CUtensorMap tm_bhi, const __grid_constant__ CUtensorMap tm_blo, Params p) {
  using C = Cfg<MODE, MH, NACC>;
  constexpr int STAGES = C::STAGES;
  if (p.gate && *p.gate == 0) return;  // uniform: another pass produces F
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint64_t* tfull = reinterpret_cast<uint64_t*>(smem + STAGES * C::STAGE_BYTES);
  uint64_t* full = tfull + STAGES;
  uint64_t* empty = full + STAGES;
  uint64_t* accf = empty + STAGES;  // [NACC]
  uint64_t* acce = accf + NACC;     // [NACC]
  uint64_t* drain = acce + NACC;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(drain + 1);
  int* abort_flag = reinterpret_cast<int*>(tmem_slot + 1);

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int units = p.tiles * p.chunks;

  if (tid == 0) {
    for (int s = 0; s < STAGES; ++s) {
      ptx::mbar_init(&tfull[s], 1);
      ptx::mbar_init(&full[s], C::CONV ? C::CW : 1);
      ptx::mbar_init(&empty[s], 1);
    }
    for (int b = 0; b < NACC; ++b) {
      ptx::mbar_init(&accf[b], 1);
      ptx::mbar_init(&acce[b], C::EW_N);
    }
    ptx::mbar_init(drain, 1);
    *abort_flag = 0;
    ptx::fence_mbar_init();
  }
  if (warp == C::MMA_W) ptx::tmem_alloc(tmem_slot, C::TMEM_COLS);
  ptx::tc_fence_before();
  __syncthreads();
  ptx::tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  const uint32_t sbase = ptx::smem_u32(smem);

  auto fail = [&]() {
    atomicOr(p.status, ST_TIMEOUT);
    atomicExch(abort_flag, 1);
  };
  auto aborted = [&]() { return *(volatile int*)abort_flag != 0; };
  // Rows of a unit: its chunk's BK-row blocks, interleaved with the other
  // chunks' blocks so that all CTAs stream nearby rows of X at any moment.
  auto unit_steps = [&](int64_t u) -> int64_t {
    const int64_t ch = u / p.tiles;
    return ch < p.nblocks ? (p.nblocks - ch + p.chunks - 1) / p.chunks : 0;
  };
  auto step_row = [&](int64_t u, int64_t t) -> int64_t { return (u / p.tiles + t * p.chunks) * BK; };

  if (warp == C::PROD_W) {
    // ------------------------------------------------------------ producer
    int64_t step = 0;
    bool ok = true;
    for (int64_t unit = blockIdx.x; unit < units && ok; unit += gridDim.x) {
      const int64_t nsteps = unit_steps(unit);
      const int col0 = (int)(unit % p.tiles) * C::BN;
      for (int64_t t = 0; t < nsteps; ++t, ++step) {
        const int s = (int)(step % STAGES);
        const uint32_t ph = (uint32_t)((step / STAGES) & 1);
        int good = 1;
        if (lane == 0) {
          if (!ptx::mbar_wait(&empty[s], ph ^ 1u, kWaitNs)) {
            fail();
            good = 0;
          } else if (aborted()) {
            good = 0;
          }
        }
        good = __shfl_sync(0xffffffffu, good, 0);
        if (!good) {
          ok = false;
          break;
        }
        if (lane == 0) {
          const uint32_t st = sbase + s * C::STAGE_BYTES;
          const int y = (int)step_row(unit, t);
          ptx::mbar_arrive_expect_tx(&tfull[s], C::TX);
#pragma unroll
          for (int b = 0; b < 2 * MH; ++b) {
            ptx::tma_load_2d(st + b * C::BOX, &tm_ahi, 64 * b, y, &tfull[s]);
            ptx::tma_load_2d(st + C::A_BYTES + b * C::BOX, &tm_alo, 64 * b, y, &tfull[s]);
          }
          if (!C::CONV && !C::SHARE_B) {
            const uint32_t bst = st + 2 * C::A_BYTES;
#pragma unroll
            for (int b = 0; b < C::BN / 64; ++b) {
              ptx::tma_load_2d(bst + b * C::BOX, &tm_bhi, col0 + 64 * b, y, &tfull[s]);
              if (C::NB == 2) ptx::tma_load_2d(bst + C::B_BYTES + b * C::BOX, &tm_blo, col0 + 64 * b, y, &tfull[s]);
            }
          }
        }
      }
    }
    // bounded wait for the copies of the last stages issued (already complete
    // on the normal path; in flight when the kernel aborted)
    if (lane == 0) {
      for (int64_t w = step - 1; w >= 0 && w >= step - STAGES; --w)
        ptx::mbar_wait(&tfull[w % STAGES], (uint32_t)((w / STAGES) & 1), kDrainNs);
    }
    __syncwarp();
  } else if (warp < C::CW) {
    // ------------------------------------------------------------ converters
    float sb = 1.f;
    if (MODE == M_F32) sb = pow2_scale(*p.amax_b);
    // Per-thread byte offsets of its B_VEC 16-byte loads inside a step's
    // BK x BN block (kr rows down, mn elements across), fixed for the kernel.
    constexpr int EPV = 16 / C::ELEM;  // elements per 16-byte load
    const int64_t row_bytes = p.ldb * C::ELEM;
    // Load cursor: unit lu, its step lk of lsteps, the block's first row and column.
    int64_t lu = blockIdx.x, lk = 0, lsteps = 0, lrow = 0, lcol = 0;
    bool lcols_full = true;
    auto enter_unit = [&]() {
      lk = 0;
      if (lu >= units) return;
      lsteps = unit_steps(lu);
      lrow = (lu / p.tiles) * BK;
      lcol = (lu % p.tiles) * C::BN;
      lcols_full = lcol + C::BN <= p.nb;
    };
    enter_unit();
    auto issue = [&](uint4 (&r)[C::B_VEC]) {
      const uint8_t* base = (const uint8_t*)p.X + lrow * row_bytes + lcol * C::ELEM;
      if (lcols_full && lrow + BK <= p.m) {
#pragma unroll
        for (int q = 0; q < C::B_VEC; ++q) {
          const int f = tid + C::CT * q;
          const int kr = f / (C::BN / EPV), mn = (f % (C::BN / EPV)) * EPV;
          r[q] = ldg16(base + kr * row_bytes + mn * C::ELEM);
        }
      } else {
#pragma unroll
        for (int q = 0; q < C::B_VEC; ++q) {
          const int f = tid + C::CT * q;
          const int kr = f / (C::BN / EPV), mn = (f % (C::BN / EPV)) * EPV;
          if (lrow + kr < p.m && lcol + mn < p.nb)
            r[q] = ldg16(base + kr * row_bytes + mn * C::ELEM);
          else
            r[q] = make_uint4(0u, 0u, 0u, 0u);
        }
      }
      lrow += (int64_t)p.chunks * BK;
      if (++lk >= lsteps) {
        lu += gridDim.x;
        enter_unit();
      }
    };
    auto store = [&](uint32_t stage_addr, const uint4 (&r)[C::B_VEC]) {
      const uint32_t b_hi = stage_addr + 2 * C::A_BYTES, b_lo = b_hi + C::B_BYTES;
#pragma unroll
      for (int q = 0; q < C::B_VEC; ++q) {
        const int f = tid + C::CT * q;
        if (MODE == M_F32) {
          const int kr = f / (C::BN / 4), mn = (f % (C::BN / 4)) * 4;
          const float4 v = *reinterpret_cast<const float4*>(&r[q]);
          uint32_t h0, l0, h1, l1;
          split_h2(v.x * sb, v.y * sb, h0, l0);
          split_h2(v.z * sb, v.w * sb, h1, l1);
          const uint32_t off = ptx::mn_sw128_offset(kr, mn, C::SBO_B);
          sts64(b_hi + off, h0, h1);
          sts64(b_lo + off, l0, l1);
        } else {
          // E4M3 values widen exactly to BF16
          const int kr = f / (C::BN / 16), mn = (f % (C::BN / 16)) * 16;
          const __nv_fp8_e4m3* e8 = reinterpret_cast<const __nv_fp8_e4m3*>(&r[q]);
          uint32_t w[8];
#pragma unroll
          for (int u = 0; u < 8; ++u) w[u] = pack_b2(float(e8[2 * u]), float(e8[2 * u + 1]));
          sts128(b_hi + ptx::mn_sw128_offset(kr, mn, C::SBO_B), make_uint4(w[0], w[1], w[2], w[3]));
          sts128(b_hi + ptx::mn_sw128_offset(kr, mn + 8, C::SBO_B), make_uint4(w[4], w[5], w[6], w[7]));
        }
      }
    };
    // NBUF register buffers in rotation: the loads of step t + NBUF - 1 are
    // issued before step t is converted and consumed NBUF - 1 iterations
    // later (a register copy out of a prefetch buffer would instead wait for
    // its loads at once).
    int64_t total = 0;  // steps of this CTA over all its units
    for (int64_t u = blockIdx.x; u < units; u += gridDim.x) total += unit_steps(u);
    int64_t step = 0;
    auto body = [&](uint4 (&cur)[C::B_VEC], uint4 (&nx)[C::B_VEC]) -> bool {
      if (step + C::NBUF - 1 < total) issue(nx);
      const int s = (int)(step % STAGES);
      const uint32_t ph = (uint32_t)((step / STAGES) & 1);
      if (!ptx::mbar_wait(&empty[s], ph ^ 1u, kWaitNs)) {
        fail();
        return false;
      }
      if (aborted()) return false;
      store(sbase + s * C::STAGE_BYTES, cur);
      ptx::fence_proxy_async_smem();
      __syncwarp();
      if (lane == 0) ptx::mbar_arrive(&full[s]);
      return ++step < total;
    };
    uint4 b0[C::B_VEC], b1[C::B_VEC];
    if constexpr (C::NBUF == 3) {
      uint4 b2[C::B_VEC];
      if (total > 0) issue(b0);
      if (total > 1) issue(b1);
      if (total > 0) {
        while (body(b0, b2) && body(b1, b0) && body(b2, b1)) {
        }
      }
    } else {
      if (total > 0) issue(b0);
      if (total > 0) {
        while (body(b0, b1) && body(b1, b0)) {
        }
      }
    }
  } else if (warp == C::MMA_W) {
    // ------------------------------------------------------------ MMA issuer
    if (lane == 0) {
      constexpr uint32_t idesc = ptx::idesc_f16(C::F16 ? 0 : 1, 128, C::BN, 1, 1);
      int64_t step = 0, seg = 0;
      bool ok = true;
      for (int64_t unit = blockIdx.x; unit < units && ok; unit += gridDim.x) {
        const int64_t nsteps = unit_steps(unit);
        for (int64_t t = 0; t < nsteps && ok; ++t, ++step) {
          const bool seg_start = (t % C::SEG) == 0;
          const int ab = (int)(seg % NACC);
          if (seg_start) {
            // wait until the epilogue has folded the segment that last used buffer ab
            if (!ptx::mbar_wait(&acce[ab], (uint32_t)(((seg / NACC) & 1) ^ 1), kWaitNs)) {
              fail();
              ok = false;
              break;
            }
            ptx::tc_fence_after();
          }
          const int s = (int)(step % STAGES);
          const uint32_t ph = (uint32_t)((step / STAGES) & 1);
          bool got = ptx::mbar_wait(&tfull[s], ph, kWaitNs);
          if (got && C::CONV) got = ptx::mbar_wait(&full[s], ph, kWaitNs);
          if (!got || aborted()) {
            if (!aborted()) fail();
            ok = false;
            break;
          }
          ptx::tc_fence_after();
          const uint32_t st = sbase + s * C::STAGE_BYTES;
          const uint32_t a_hi = st, b_hi = C::SHARE_B ? st : st + 2 * C::A_BYTES;
          // descriptors of the stage's operands; K slices and M halves are offsets
          const uint64_t adh0 = ptx::desc_sw128(a_hi, C::BOX, 1024);
          const uint64_t bdh0 = C::CONV ? ptx::desc_sw128(b_hi, 1024, C::SBO_B) : ptx::desc_sw128(b_hi, C::BOX, 1024);
          constexpr uint32_t B_KSTEP = C::CONV ? 2 * C::SBO_B : 2048;  // bytes per 16 K-rows of B
#pragma unroll
          for (int kk = 0; kk < BK / 16; ++kk) {
            const uint64_t bdh = ptx::desc_advance(bdh0, kk * B_KSTEP);
            const uint64_t bdl = ptx::desc_advance(bdh, C::SHARE_B ? C::A_BYTES : C::B_BYTES);
#pragma unroll
            for (int h = 0; h < MH; ++h) {
              const uint32_t d = tmem + (uint32_t)(ab * C::ACC_COLS + h * C::BN);
              const uint64_t adh = ptx::desc_advance(adh0, h * 2 * C::BOX + kk * 2048);
              const uint64_t adl = ptx::desc_advance(adh, C::A_BYTES);
              const uint32_t acc = (seg_start && kk == 0) ? 0u : 1u;
              ptx::mma_f16(d, adh, bdh, idesc, acc);
              if (C::NB == 2) ptx::mma_f16(d, adh, bdl, idesc, 1u);
              ptx::mma_f16(d, adl, bdh, idesc, 1u);
            }
          }
          ptx::mma_commit(&empty[s]);
          if ((t % C::SEG) == C::SEG - 1 || t == nsteps - 1) {
            ptx::mma_commit(&accf[ab]);
            ++seg;
          }
        }
      }
      // drain: every MMA issued by this thread completes before TMEM is freed
      ptx::mma_commit(drain);
      if (!ptx::mbar_wait(drain, 0u, kWaitNs)) atomicOr(p.status, ST_TIMEOUT);
    }
    __syncwarp();
  } else {
    // ------------------------------------------------------------ epilogue
    const int e = (warp - C::EPI0) & 3;       // TMEM lane quarter
    const int ehalf = (warp - C::EPI0) >> 2;  // which half of the columns this warp folds
    float sc = 1.f;
    if (MODE == M_F32) sc = 1.f / (pow2_scale(*p.amax_u) * pow2_scale(*p.amax_b));
    if (MODE == M_GRAM) sc = 1.f / (pow2_scale(*p.amax_u) * pow2_scale(*p.amax_u));
    const uint32_t lane_base = (uint32_t)(32 * e) << 16;
    constexpr int EW = C::CW > 8 ? 16 : 32;  // TMEM columns per fold chunk (registers are scarcer with 16 converters)
    int64_t seg = 0;
    bool ok = true;
    for (int64_t unit = blockIdx.x; unit < units && ok; unit += gridDim.x) {
      const int tile = (int)(unit % p.tiles);
      const int64_t ch = unit / p.tiles;
      const int64_t nsteps = unit_steps(unit);
      const int64_t nseg = (nsteps + C::SEG - 1) / C::SEG;
      for (int64_t g = 0; g < nseg; ++g, ++seg) {
        const int ab = (int)(seg % NACC);
        if (!ptx::mbar_wait(&accf[ab], (uint32_t)((seg / NACC) & 1), kWaitNs) || aborted()) {
          if (!aborted()) fail();
          ok = false;
          break;
        }
        ptx::tc_fence_after();
        const bool first = g == 0, last = g == nseg - 1;
        const uint32_t abase = tmem + lane_base + (uint32_t)(ab * C::ACC_COLS);
        const uint32_t sbase_t = tmem + lane_base + C::S_COL;
#pragma unroll
        for (int h = 0; h < MH; ++h) {
          const int c = 128 * h + 32 * e + lane;
#pragma unroll 1
          for (int cc = ehalf * (C::BN / 2); cc < (ehalf + 1) * (C::BN / 2); cc += EW) {
            const uint32_t col = (uint32_t)(h * C::BN + cc);
            uint32_t a[EW], r[EW];
            // the previous chunk's store of S has to land before r is reloaded
            ptx::tmem_wait_st(r);
            if constexpr (EW == 32) {
              ptx::tmem_ld32_nowait(abase + col, a);
              if (!first) ptx::tmem_ld32_nowait(sbase_t + col, r);
            } else {
              ptx::tmem_ld16_nowait(abase + col, a);
              if (!first) ptx::tmem_ld16_nowait(sbase_t + col, r);
            }
            ptx::tmem_wait_ld(a);
            if (first) {
#pragma unroll
              for (int q = 0; q < EW; ++q) r[q] = a[q];
            } else {
              ptx::tmem_regs_ready(r);
#pragma unroll
              for (int q = 0; q < EW; ++q) r[q] = __float_as_uint(__uint_as_float(r[q]) + __uint_as_float(a[q]));
            }
            if (!last) {
              if constexpr (EW == 32) ptx::tmem_st32_nowait(sbase_t + col, r);
              else ptx::tmem_st16_nowait(sbase_t + col, r);
            } else if (c < p.k) {
              const int64_t j0 = (int64_t)tile * C::BN + cc;
              float* dst = p.part + (ch * p.k + c) * p.nb + j0;
              if (j0 + EW <= p.nb && (p.nb & 3) == 0) {
#pragma unroll
                for (int q = 0; q < EW; q += 4)
                  *reinterpret_cast<float4*>(dst + q) =
                      make_float4(__uint_as_float(r[q]) * sc, __uint_as_float(r[q + 1]) * sc,
                                  __uint_as_float(r[q + 2]) * sc, __uint_as_float(r[q + 3]) * sc);
              } else {
#pragma unroll
                for (int q = 0; q < EW; ++q)
                  if (j0 + q < p.nb) dst[q] = __uint_as_float(r[q]) * sc;
              }
            }
          }
        }
        ptx::tc_fence_before();
        __syncwarp();
        if (lane == 0) ptx::mbar_arrive(&acce[ab]);
      }
    }
    ptx::tmem_wait_st();
  }

  __syncthreads();
  if (warp == C::MMA_W) {
    ptx::tc_fence_after();
    ptx::tmem_dealloc(tmem, C::TMEM_COLS);
  }
}

// about four units per CTA, chunks of >= 512 rows, a multiple of BK rows
// About `per_sm` units per SM (tiles x chunks), chunks of at least 512 rows.
void choose_chunks(int64_t m, int tiles, int num_sms, int& chunks, int64_t& rows, int per_sm = 4) {
  int64_t c = ((int64_t)per_sm * num_sms + tiles - 1) / tiles;
  const int64_t cmax = (m + 511) / 512;
  if (c > cmax) c = cmax;
  if (c < 1) c = 1;
  rows = (m + c - 1) / c;
  rows = (rows + BK - 1) / BK * BK;
  chunks = (int)((m + rows - 1) / rows);
}

template <int MODE, int MH, int NACC>
bool launch(Launcher& L, const CUtensorMap& ahi, const CUtensorMap& alo, const CUtensorMap& bhi,
            const CUtensorMap& blo, const Params& p) {
  using C = Cfg<MODE, MH, NACC>;
  if (cudaFuncSetAttribute(passf_kernel<MODE, MH, NACC>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)C::SMEM) != cudaSuccess)
    return false;
  const int units = p.tiles * p.chunks;
  const int grid = units < L.num_sms ? units : L.num_sms;
  passf_kernel<MODE, MH, NACC><<<grid, C::THREADS, C::SMEM, L.stream>>>(ahi, alo, bhi, blo, p);
  L.count(1);
  return true;
}

// k <= 128: one 256-column accumulator; k > 128: two M halves of 128 columns.
// (NACC = 2 -- 128-column tiles with a double-buffered accumulator, so the
// tensor core never waits for the fold -- measured slower on GB300 at
// 200,000 x 4,096: twice the MMA instructions and the U copies per X byte.)
int tile_cols(int k) { return k > 128 ? 128 : 256; }

template <int MODE>
bool launch_k(Launcher& L, int k, const CUtensorMap& ahi, const CUtensorMap& alo, const CUtensorMap& bhi,
              const CUtensorMap& blo, const Params& p) {
  if (k > 128) return launch<MODE, 2, 1>(L, ahi, alo, bhi, blo, p);
  // the Gram's 128-column tile leaves TMEM room for a second accumulator
  if constexpr (MODE == M_GRAM) return launch<MODE, 1, 2>(L, ahi, alo, bhi, blo, p);
  else return launch<MODE, 1, 1>(L, ahi, alo, bhi, blo, p);
}

int64_t pitch16(int k) { return ((int64_t)k + 7) / 8 * 8; }

}  // namespace pf

void plan_tc_chain(char* base, TcChainWs& w, int xt, int64_t m, int64_t n, int k, bool want_g, int num_sms) {
  const int BN = pf::tile_cols(k);
  const int tiles = (int)((n + BN - 1) / BN);
  int chunks;
  int64_t rows;
  pf::choose_chunks(m, tiles, num_sms, chunks, rows);
  w.chunks = chunks;
  w.rows_per_chunk = rows;
  w.ku = pf::pitch16(k);
  size_t off = 0;
  auto take = [&](size_t b) {
    off = (off + 255) & ~(size_t)255;
    char* r = base ? base + off : nullptr;
    off += b;
    return r;
  };
  const size_t split_bytes = (size_t)m * (size_t)w.ku * 2;
  w.Fpart = (double*)take((size_t)chunks * k * n * 4);  // FP32 partials (typed as bytes)
  w.uhi = take(split_bytes);
  w.ulo = take(split_bytes);
  w.Gpart = nullptr;
  w.ghi = w.glo = nullptr;
  w.gchunks = 0;
  if (want_g) {
    const int gt = (k + BN - 1) / BN;
    int gc;
    int64_t grows;
    // one unit per SM: the Gram has a single tile, so short chunks would each
    // pay the pipeline's fill and drain and write a k x k partial
    pf::choose_chunks(m, gt, num_sms, gc, grows, 1);
    w.gchunks = gc;
    w.grows_per_chunk = grows;
    w.Gpart = (double*)take((size_t)gc * k * k * 4);
    if (xt != LSPCA_F32) {
      // the Gram takes FP16 pairs; BF16 / E4M3 X split U into BF16 pairs for F
      w.ghi = take(split_bytes);
      w.glo = take(split_bytes);
    }
  }
  w.bytes = off + 256;
}

bool tc_chain_main(Launcher& L, const void* X, int xt, int64_t m, int64_t n, int64_t ldx, const float* U, int k,
                   TcChainWs& w, const float* absmax, int* status, bool want_g, const int* gate) {
  const int BN = pf::tile_cols(k);
  const bool f16 = xt == LSPCA_F32;
  const int threads = 256;
  const int64_t total4 = m * (k / 4);
  int blocks = (int)((total4 + threads - 1) / threads);
  if (blocks > 8 * L.num_sms) blocks = 8 * L.num_sms;
  if (f16)
    pf::split_u_kernel<true><<<blocks, threads, 0, L.stream>>>(U, m, k, w.ku, absmax + 1, (uint16_t*)w.uhi,
                                                                (uint16_t*)w.ulo, gate);
  else
    pf::split_u_kernel<false><<<blocks, threads, 0, L.stream>>>(U, m, k, w.ku, absmax + 1, (uint16_t*)w.uhi,
                                                                 (uint16_t*)w.ulo, gate);
  L.count(1);
  const CUtensorMapDataType adt = f16 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT16 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16;
  CUtensorMap ahi, alo, bhi, blo;
  if (!make_tmap_2d_sw128(&ahi, w.uhi, adt, 2, (uint64_t)m, (uint64_t)k, (uint64_t)w.ku * 2, pf::BK, 64) ||
      !make_tmap_2d_sw128(&alo, w.ulo, adt, 2, (uint64_t)m, (uint64_t)k, (uint64_t)w.ku * 2, pf::BK, 64))
    return false;
  bhi = ahi;
  blo = alo;
  if (xt == LSPCA_BF16 &&
      !make_tmap_2d_sw128(&bhi, X, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, (uint64_t)m, (uint64_t)n, (uint64_t)ldx * 2,
                          pf::BK, 64))
    return false;
  pf::Params p{};
  p.X = X;
  p.ldb = ldx;
  p.nb = n;
  p.m = m;
  p.k = k;
  p.tiles = (int)((n + BN - 1) / BN);
  p.chunks = w.chunks;
  p.nblocks = (m + pf::BK - 1) / pf::BK;
  p.part = (float*)w.Fpart;
  p.amax_b = absmax;
  p.amax_u = absmax + 1;
  p.status = status;
  p.gate = gate;
  bool ok;
  if (xt == LSPCA_F32) ok = pf::launch_k<pf::M_F32>(L, k, ahi, alo, bhi, blo, p);
  else if (xt == LSPCA_BF16) ok = pf::launch_k<pf::M_BF16>(L, k, ahi, alo, bhi, blo, p);
  else ok = pf::launch_k<pf::M_E4M3>(L, k, ahi, alo, bhi, blo, p);
  if (!ok) return false;
  if (want_g) {
    // G = U^T U from FP16 pairs of U (the F pairs when X is FP32)
    CUtensorMap ghi = ahi, glo = alo;
    if (xt != LSPCA_F32) {
      pf::split_u_kernel<true><<<blocks, threads, 0, L.stream>>>(U, m, k, w.ku, absmax + 1, (uint16_t*)w.ghi,
                                                                  (uint16_t*)w.glo, nullptr);
      L.count(1);
      if (!make_tmap_2d_sw128(&ghi, w.ghi, CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 2, (uint64_t)m, (uint64_t)k,
                              (uint64_t)w.ku * 2, pf::BK, 64) ||
          !make_tmap_2d_sw128(&glo, w.glo, CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 2, (uint64_t)m, (uint64_t)k,
                              (uint64_t)w.ku * 2, pf::BK, 64))
        return false;
    }
    pf::Params g = p;
    g.gate = nullptr;
    g.X = nullptr;
    g.nb = k;
    g.tiles = (k + BN - 1) / BN;
    g.chunks = w.gchunks;

    g.part = (float*)w.Gpart;
    g.amax_b = absmax + 1;
    if (!pf::launch_k<pf::M_GRAM>(L, k, ghi, glo, ghi, glo, g)) return false;
  }
  return true;
}

}  // namespace lspca
