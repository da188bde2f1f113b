// TMA-fed tensor-core reduction map Y = X V (Sec. III-B.2: pi(x) = V^T x for
// every row) for BF16 and FP8 E4M3 X on sm_103a; with V = the BF16-rounded
// Gaussian Omega the same kernel computes the sketch U = X Omega (Eq. 1).
//
// GEMM view: M = 128 rows of X per tile, N = k padded to a multiple of 64
// (NPAD), K = n in k-steps of 64.  A = the X tile (K-major), B = V (MN-major,
// pre-split and pre-swizzled per k-step by tile_v_kernel).
//
// Why a second kernel next to tcproj.cu's: there the X rows pass through the
// registers of converter warps, two k-steps ahead, and the loads' latency
// bounds the kernel (most warp samples stall on the load scoreboard).  Here
// X arrives by TMA (cp.async.bulk.tensor, 128-byte swizzle) into a ring of
// shared-memory stages issued by one thread as far ahead as the ring allows.
//
// Number formats.
// * BF16 X: the TMA box is the A operand as it stands.  V is split into a
//   BF16 pair v = hi + lo (two products), or taken as one exact piece (the
//   BF16-rounded Omega of the sketch, one product).
// * E4M3 X: every E4M3 value is exact in FP16, so converter warps widen each
//   128-byte TMA box (two k-steps) into two FP16 A tiles, shared memory to
//   shared memory (cvt.rn.f16x2.e4m3x2, no rounding).  V is split into an
//   FP16 pair of V t (t a power of two from max|V|), two products, and the
//   epilogue multiplies by 1 / t (exact).  The pair keeps 22 significant bits.
//
// Accumulation.  tcgen05.mma's FP32 accumulation truncates, so the tensor
// core accumulates segments of SEG k-steps into a TMEM accumulator and the
// epilogue folds each into a round-to-nearest FP32 running sum S in TMEM,
// writing S as the rows of Y after the last segment.  For NPAD <= 128 two
// accumulators alternate, so the tensor core runs on while a fold is read.
//
// CTA pairs.  The kernel runs in clusters of two CTAs on neighbouring SMs
// that take consecutive row tiles and share every V stage: each CTA fetches
// half of the stage and multicasts it into both (cp.async.bulk
// .multicast::cluster), and each MMA thread signals the stage free in both
// CTAs (tcgen05.commit .multicast::cluster), so every SM pulls half as much V
// out of L2 and its TMA unit issues half the copies.  Both CTAs walk K in the
// same order, rotated per pair.
//
// Roles (one persistent CTA per SM):
//   warps 0..CW-1       converters (E4M3 only, CW = 2);
//   warps CW..CW+7      epilogue: two per TMEM lane quarter (the quarter is
//                       the warp index mod 4), each folding half the columns;
//   warp  CW+8          TMEM allocation and the thread that issues tcgen05.mma;
//   warp  CW+9          producer: TMA of X, bulk copies of V tiles.
// Every wait is bounded (2 s of %globaltimer): on expiry the kernel records
// ST_TIMEOUT and raises the CTA's abort flag; every role leaves its loop, the
// producer waits (bounded) for its copies in flight, the MMA thread for its
// products, and TMEM is freed.
#include <cuda_fp16.h>
#include <cuda_fp8.h>

#include "common.cuh"
#include "tc.h"
#include "tc_ptx.cuh"
#include "tma.h"

namespace lspca {
namespace xp {

constexpr int BK = 64;                      // K per k-step (one 128-byte row of 16-bit A)
constexpr uint32_t A_BYTES = 128 * BK * 2;  // one A tile: 16 KB
constexpr uint32_t RAW_BYTES = 128 * 128;   // one E4M3 box: 128 rows x 128 bytes (two k-steps)
constexpr uint64_t kWaitNs = 2000000000ull;
constexpr uint64_t kDrainNs = 100000000ull;
// k-steps per accumulation segment: 8 where two accumulators alternate; 16
// where one 256-column accumulator must wait for each fold's loads (k > 128)
constexpr int SEG2 = 8, SEG1 = 16;
constexpr int kSmemBudget = 220 * 1024;

struct Params {
  int64_t m, n;
  int k;
  int64_t tiles;        // 128-row tiles
  int nks;              // k-steps of 64
  const uint8_t* vt;    // V tiles: per k-step [hi | lo], each BK x NPAD 16-bit, MN-major SW128
  const float* vscale;  // E4M3: device t (V t was split); nullptr = 1
  float* Y;             // m x k FP32
  float* ymax;          // nullable: max|Y|
  int check_y;          // non-finite Y sets ST_NONFINITE
  int* status;
};

template <bool E4M3, int NT, bool EXACT_V>
struct Cfg {
  static constexpr int NPAD = 64 * NT;
  static constexpr int PB = EXACT_V ? 1 : 2;                 // V pieces
  static constexpr uint32_t B_BYTES = BK * NPAD * 2;         // one piece of one k-step
  static constexpr uint32_t SBO_B = NT * 1024;
  // V arrives in stages of B_SUB K-slices (16 K-rows each) of every piece, at
  // least 32 KB a stage: small stages keep more of V in flight per byte of ring
  static constexpr uint32_t SLICE = 2 * SBO_B;               // one K-slice of one piece
  static constexpr int B_SUB0 = (int)(32768 / (PB * SLICE));
  static constexpr int B_SUB = B_SUB0 < 1 ? 1 : (B_SUB0 > 4 ? 4 : B_SUB0);
  static constexpr int SUBS = (BK / 16) / B_SUB;              // V stages per k-step
  static constexpr uint32_t B_PART = B_SUB * SLICE;           // one piece of one stage
  static constexpr uint32_t B_STAGE = PB * B_PART;
  static constexpr int CW = E4M3 ? 2 : 0;                    // converter warps
  static constexpr int EPI0 = CW;
  static constexpr int EW = 8;                               // epilogue warps
  static constexpr int MMA_W = CW + EW;
  static constexpr int PROD_W = CW + EW + 1;
  static constexpr int THREADS = (CW + EW + 2) * 32;
  // rings: E4M3 raw boxes (two k-steps each), A tiles and V tiles (one k-step each)
  static constexpr int R_STAGES = E4M3 ? 2 : 0;
  static constexpr int A_STAGES = E4M3 ? 3 : 4;
  static constexpr int CWX = CW > 0 ? CW : 1;               // divisors for the converter code,
  static constexpr int RSX = R_STAGES > 0 ? R_STAGES : 1;   // which BF16 instances never run
  static constexpr uint32_t FIXED = R_STAGES * RAW_BYTES + A_STAGES * A_BYTES;
  static constexpr int B_STAGES_FIT = (int)((kSmemBudget - FIXED) / B_STAGE);
  static constexpr int B_STAGES = B_STAGES_FIT > 8 ? 8 : B_STAGES_FIT;
  static constexpr int NACC = NPAD <= 128 ? 2 : 1;
  static constexpr int SEG = NACC == 2 ? SEG2 : SEG1;
  static constexpr uint32_t S_COL = NACC * NPAD;
  static constexpr uint32_t TMEM_COLS = S_COL + NPAD <= 256 ? 256 : 512;
  static constexpr int WCOLS = NPAD / 2;                     // columns folded per epilogue warp
  static constexpr int NCH = WCOLS / 32;
  static constexpr size_t SMEM = 1024 + (size_t)FIXED + (size_t)B_STAGES * B_STAGE + 512;
  static_assert(B_STAGES >= 2, "shared-memory budget");
  static_assert(R_STAGES <= 4 && A_STAGES <= 4 && B_STAGES <= 8, "barrier slots");
  static_assert(SUBS * B_SUB == BK / 16, "V stages tile the k-step");
  static_assert(S_COL + NPAD <= 512, "TMEM budget");
  static_assert(WCOLS % 32 == 0, "fold chunks of 32 columns");
};

// Bounded wait; on expiry the status and the CTA's abort flag are set.
__device__ __forceinline__ bool wait_or_abort(uint64_t* bar, uint32_t parity, volatile int* abort, int* status) {
  if (*abort) return false;
  if (ptx::mbar_wait(bar, parity, kWaitNs)) return true;
  *abort = 1;
  atomicOr(status, ST_TIMEOUT);
  return false;
}

// The same wait taken by every lane of a warp, with a warp-uniform outcome:
// lanes whose waits end on either side of the limit still leave together.
__device__ __forceinline__ bool warp_wait(uint64_t* bar, uint32_t parity, volatile int* abort, int* status) {
  const bool ok = wait_or_abort(bar, parity, abort, status);
  return __all_sync(0xffffffffu, ok);
}

// The X box (and its V tiles) taken j-th: every CTA pair walks K in its own
// rotation, (tile / 2) mod boxes, so the pairs, which hold consecutive tiles,
// read different V tiles at any moment instead of all loading the same one
// from the same L2 slices.  A row's result depends only on its tile.
__device__ __forceinline__ int box_rotation(int64_t t, int nboxes) { return (int)(t % nboxes); }
__device__ __forceinline__ int rotated_box(int rot, int j, int nboxes) {
  const int b = j + rot;
  return b >= nboxes ? b - nboxes : b;
}

// Four E4M3 bytes (K order, low byte first) -> two words of FP16 pairs, exact.
__device__ __forceinline__ void e4m3x4_to_f16(uint32_t w, uint32_t& lo, uint32_t& hi) {
  asm("{\n\t.reg .b16 l, h;\n\t"
      "mov.b32 {l, h}, %2;\n\t"
      "cvt.rn.f16x2.e4m3x2 %0, l;\n\t"
      "cvt.rn.f16x2.e4m3x2 %1, h;\n\t}"
      : "=r"(lo), "=r"(hi)
      : "r"(w));
}

template <bool E4M3, int NT, bool EXACT_V>
__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(Cfg<E4M3, NT, EXACT_V>::THREADS, 1)
    xproj_kernel(const __grid_constant__ CUtensorMap tmx, Params p) {
  using C = Cfg<E4M3, NT, EXACT_V>;
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint8_t* raw = smem;                                           // [R_STAGES][RAW_BYTES]
  uint8_t* atile = raw + C::R_STAGES * RAW_BYTES;                // [A_STAGES][A_BYTES]
  uint8_t* btile = atile + C::A_STAGES * A_BYTES;                // [B_STAGES][B_STAGE]
  uint64_t* bars = (uint64_t*)(btile + (size_t)C::B_STAGES * C::B_STAGE);
  uint64_t* rfull = bars;
  uint64_t* rempty = rfull + 4;
  uint64_t* afull = rempty + 4;
  uint64_t* aempty = afull + 4;
  uint64_t* bfull = aempty + 4;
  uint64_t* bempty = bfull + 8;
  uint64_t* accf = bempty + 8;  // [NACC]
  uint64_t* acce = accf + 2;    // [NACC]
  uint64_t* drain = acce + 2;
  uint32_t* tslot = (uint32_t*)(drain + 1);
  volatile int* abort = (volatile int*)(tslot + 1);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nks = p.nks;
  const int nboxes = E4M3 ? (nks + 1) / 2 : nks;  // X boxes per tile

  if (threadIdx.x == 0) {
    for (int s = 0; s < C::R_STAGES; ++s) {
      ptx::mbar_init(&rfull[s], 1);
      ptx::mbar_init(&rempty[s], C::CW);
    }
    for (int s = 0; s < C::A_STAGES; ++s) {
      ptx::mbar_init(&afull[s], E4M3 ? C::CW : 1);  // converter warps, or the producer's expect-tx
      ptx::mbar_init(&aempty[s], 1);
    }
    for (int s = 0; s < C::B_STAGES; ++s) {
      ptx::mbar_init(&bfull[s], 1);
      ptx::mbar_init(&bempty[s], 2);  // both CTAs of the pair have consumed the stage
    }
    for (int b = 0; b < C::NACC; ++b) {
      ptx::mbar_init(&accf[b], 1);
      ptx::mbar_init(&acce[b], C::EW);
    }
    ptx::mbar_init(drain, 1);
    *abort = 0;
    ptx::fence_mbar_init();
  }
  if (warp == C::MMA_W) ptx::tmem_alloc(tslot, C::TMEM_COLS);
  ptx::tc_fence_before();
  __syncthreads();
  ptx::tc_fence_after();
  const uint32_t tmem = *tslot;
  // the pair's barriers exist before either CTA multicasts into the other
  ptx::cluster_sync();
  // A CTA pair takes tiles t0 and t0 + 1 (t0 even); both run the same number
  // of pair steps (a tile past the end is a phantom: TMA fills zeros, nothing
  // is written) and walk K in the pair's rotation.
  const int crank = (int)ptx::cluster_ctarank();
  const int64_t t0_first = (int64_t)blockIdx.x - crank;

  if (warp == C::PROD_W) {
    // ------------------------------------------------------------ producer
    // Two cursors, X boxes and V tiles, each issued as soon as its ring has
    // a free stage (non-blocking tests), so X runs as far ahead as its ring
    // allows whatever the V ring does.
    if (lane == 0) {
      constexpr int XS = E4M3 ? C::R_STAGES : C::A_STAGES;
      constexpr uint32_t XB = E4M3 ? RAW_BYTES : A_BYTES;
      uint64_t* xf = E4M3 ? rfull : afull;
      uint64_t* xe = E4M3 ? rempty : aempty;
      uint8_t* xr = E4M3 ? raw : atile;
      const int64_t mine = p.tiles > t0_first ? (p.tiles - 1 - t0_first) / gridDim.x + 1 : 0;
      const int64_t xtot = mine * nboxes, btot = mine * nks * C::SUBS;
      // cursors kept incrementally (no divisions in the issue loop)
      int64_t xi = 0, bi = 0, xpair = t0_first, bpair = t0_first;
      int xj = 0, xs = 0, bj = 0, bh = 0, bsub = 0, bs = 0;
      int xrot = box_rotation(xpair >> 1, nboxes), brot = xrot;
      uint32_t xph = 0, bph = 0;
      uint64_t t0 = 0;  // start of the current run of polls without progress
      while (xi < xtot || bi < btot) {
        bool prog = false;
        if (xi < xtot && ptx::mbar_test_wait(&xe[xs], xph ^ 1u)) {
          ptx::mbar_arrive_expect_tx(&xf[xs], XB);
          const int xb = rotated_box(xrot, xj, nboxes);
          ptx::tma_load_2d(ptx::smem_u32(xr + (size_t)xs * XB), &tmx, xb * (E4M3 ? 128 : BK),
                           (int)((xpair + crank) * 128), &xf[xs]);
          ++xi;
          if (++xj == nboxes) {
            xj = 0;
            xpair += gridDim.x;
            xrot = box_rotation(xpair >> 1, nboxes);
          }
          if (++xs == XS) {
            xs = 0;
            xph ^= 1u;
          }
          prog = true;
        }
        if (bi < btot && ptx::mbar_test_wait(&bempty[bs], bph ^ 1u)) {
          const int bb = rotated_box(brot, bj, nboxes);
          const int bks = E4M3 ? 2 * bb + bh : bb;
          // this CTA fetches its half of the stage (piece crank, or half the
          // single piece) into both CTAs of the pair
          constexpr uint32_t HALF = C::PB == 2 ? C::B_PART : C::B_PART / 2;
          const uint8_t* src = p.vt + (size_t)bks * 2 * C::B_BYTES + (size_t)bsub * C::B_PART +
                               (C::PB == 2 ? (size_t)crank * C::B_BYTES : (size_t)crank * HALF);
          const uint32_t dst = ptx::smem_u32(btile + (size_t)bs * C::B_STAGE) + (uint32_t)crank * HALF;
          ptx::mbar_arrive_expect_tx(&bfull[bs], C::B_STAGE);
          ptx::bulk_g2s_mc(dst, src, HALF, &bfull[bs], (uint16_t)0x3);
          ++bi;
          if (++bsub == C::SUBS) {
            bsub = 0;
            // next k-step: the box's second half (E4M3, if it exists), else the next box
            if (E4M3 && bh == 0 && 2 * bb + 1 < nks) {
              bh = 1;
            } else {
              bh = 0;
              if (++bj == nboxes) {
                bj = 0;
                bpair += gridDim.x;
                brot = box_rotation(bpair >> 1, nboxes);
              }
            }
          }
          if (++bs == C::B_STAGES) {
            bs = 0;
            bph ^= 1u;
          }
          prog = true;
        }
        if (prog) {
          t0 = 0;
          continue;
        }
        if (*abort) break;
        const uint64_t now = ptx::globaltimer();
        if (t0 == 0) t0 = now;
        if (now - t0 > kWaitNs) {
          *abort = 1;
          atomicOr(p.status, ST_TIMEOUT);
          break;
        }
        __nanosleep(20);
      }
      if (*abort) {  // copies in flight land before the CTA leaves
        for (int64_t q = xi - XS; q < xi; ++q)
          if (q >= 0) ptx::mbar_wait(&xf[q % XS], (uint32_t)((q / XS) & 1), kDrainNs);
        for (int64_t q = bi - C::B_STAGES; q < bi; ++q)
          if (q >= 0) ptx::mbar_wait(&bfull[q % C::B_STAGES], (uint32_t)((q / C::B_STAGES) & 1), kDrainNs);
      }
    }
    __syncwarp();
  } else if (E4M3 && warp < C::CW) {
    // ------------------------------------------------------------ converters
    // Half h of a box (K bytes 64h .. 64h + 63) becomes the FP16 A tile of
    // k-step 2j + h.  Thread (warp w, lane l) converts, in pass i, the 16-byte
    // chunk c = 4h + (l & 3) of row r = 8 CW i + 8 w + (l >> 2) into the FP16
    // chunks 2(l & 3) and 2(l & 3) + 1 of the tile.
    const int cq = lane & 3;
    int64_t ri = 0, ai = 0;
    bool ok = true;
    for (int64_t t0 = t0_first; t0 < p.tiles && ok; t0 += gridDim.x) {
      const int rot = box_rotation(t0 >> 1, nboxes);
      for (int j = 0; j < nboxes && ok; ++j, ++ri) {
        const int rs = (int)(ri % C::RSX);
        if (!warp_wait(&rfull[rs], (uint32_t)((ri / C::RSX) & 1), abort, p.status)) {
          ok = false;
          break;
        }
        const uint32_t src = ptx::smem_u32(raw + (size_t)rs * RAW_BYTES);
        const int jb = rotated_box(rot, j, nboxes);
        for (int h = 0; h < 2 && 2 * jb + h < nks; ++h, ++ai) {
          const int as = (int)(ai % C::A_STAGES);
          if (!warp_wait(&aempty[as], (uint32_t)((ai / C::A_STAGES) & 1) ^ 1u, abort, p.status)) {
            ok = false;
            break;
          }
          const uint32_t dst = ptx::smem_u32(atile + (size_t)as * A_BYTES);
          const uint32_t c = (uint32_t)(4 * h + cq), c0 = (uint32_t)(2 * cq);
#pragma unroll
          for (int i = 0; i < 128 / (8 * C::CWX); ++i) {
            const int r = 8 * C::CWX * i + 8 * warp + (lane >> 2);
            const uint32_t sw = (uint32_t)(r & 7);
            uint32_t w0, w1, w2, w3;
            asm volatile("ld.shared.v4.u32 {%0, %1, %2, %3}, [%4];"
                         : "=r"(w0), "=r"(w1), "=r"(w2), "=r"(w3)
                         : "r"(src + (uint32_t)r * 128u + ((c ^ sw) << 4)));
            uint32_t hv[8];
            e4m3x4_to_f16(w0, hv[0], hv[1]);
            e4m3x4_to_f16(w1, hv[2], hv[3]);
            e4m3x4_to_f16(w2, hv[4], hv[5]);
            e4m3x4_to_f16(w3, hv[6], hv[7]);
            const uint32_t rowb = dst + (uint32_t)r * 128u;
            asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(rowb + ((c0 ^ sw) << 4)), "r"(hv[0]),
                         "r"(hv[1]), "r"(hv[2]), "r"(hv[3])
                         : "memory");
            asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(rowb + (((c0 + 1) ^ sw) << 4)),
                         "r"(hv[4]), "r"(hv[5]), "r"(hv[6]), "r"(hv[7])
                         : "memory");
          }
          ptx::fence_proxy_async_smem();
          __syncwarp();
          if (lane == 0) ptx::mbar_arrive(&afull[as]);
        }
        __syncwarp();
        if (lane == 0) ptx::mbar_arrive(&rempty[rs]);
      }
    }
  } else if (warp == C::MMA_W) {
    // ------------------------------------------------------------ MMA issuer
    if (lane == 0) {
      constexpr uint32_t idesc = ptx::idesc_f16(E4M3 ? 0 : 1, 128, C::NPAD, 0, 1);
      // ring cursors kept incrementally: stage index and phase parity
      int as = 0, bs = 0, ab = 0;
      uint32_t aph = 0, bph = 0, accph = 0;
      bool ok = true;
      for (int64_t t0 = t0_first; t0 < p.tiles && ok; t0 += gridDim.x) {
        for (int ks = 0; ks < nks && ok; ++ks) {
          const bool seg_start = (ks % C::SEG) == 0;
          if (seg_start) {
            // the epilogue has read the segment that last used accumulator ab
            if (!wait_or_abort(&acce[ab], accph ^ 1u, abort, p.status)) {
              ok = false;
              break;
            }
            ptx::tc_fence_after();
          }
          if (!wait_or_abort(&afull[as], aph, abort, p.status)) {
            ok = false;
            break;
          }
          ptx::tc_fence_after();
          const uint32_t a0 = ptx::smem_u32(atile + (size_t)as * A_BYTES);
          const uint32_t d = tmem + (uint32_t)(ab * C::NPAD);
          const uint64_t ad0 = ptx::desc_sw128(a0, 16, 1024);
          for (int sub = 0; sub < C::SUBS && ok; ++sub) {
            if (!wait_or_abort(&bfull[bs], bph, abort, p.status)) {
              ok = false;
              break;
            }
            ptx::tc_fence_after();
            const uint64_t bd0 = ptx::desc_sw128(ptx::smem_u32(btile + (size_t)bs * C::B_STAGE), 1024, C::SBO_B);
#pragma unroll
            for (int q = 0; q < C::B_SUB; ++q) {
              const int kk = sub * C::B_SUB + q;
              const uint64_t ad = ptx::desc_advance(ad0, kk * 32);
              const uint64_t bd = ptx::desc_advance(bd0, q * C::SLICE);
              ptx::mma_f16(d, ad, bd, idesc, (seg_start && kk == 0) ? 0u : 1u);
              if (!EXACT_V) ptx::mma_f16(d, ad, ptx::desc_advance(bd, C::B_PART), idesc, 1u);
            }
            ptx::mma_commit_mc(&bempty[bs], (uint16_t)0x3);  // the stage is free in both CTAs
            if (++bs == C::B_STAGES) {
              bs = 0;
              bph ^= 1u;
            }
          }
          if (!ok) break;
          ptx::mma_commit(&aempty[as]);
          if (++as == C::A_STAGES) {
            as = 0;
            aph ^= 1u;
          }
          if ((ks % C::SEG) == C::SEG - 1 || ks == nks - 1) {
            ptx::mma_commit(&accf[ab]);
            if (++ab == C::NACC) {
              ab = 0;
              accph ^= 1u;
            }
          }
        }
      }
      ptx::mma_commit(drain);  // all products of this thread done before TMEM is freed
      if (!ptx::mbar_wait(drain, 0u, kDrainNs)) atomicOr(p.status, ST_TIMEOUT);
    }
    __syncwarp();
  } else if (warp >= C::EPI0 && warp < C::EPI0 + C::EW) {
    // ------------------------------------------------------------ epilogue
    const int e = warp & 3;                   // TMEM lane quarter of this warp
    const int ehalf = (warp - C::EPI0) >> 2;  // which half of the columns it folds
    const uint32_t lane_base = (uint32_t)(32 * e) << 16;
    const float us = p.vscale ? 1.f / *p.vscale : 1.f;
    uint32_t yb = 0u;  // max|Y| written, as FP32 bits
    const int nseg = (nks + C::SEG - 1) / C::SEG;
    int64_t seg = 0;
    bool ok = true;
    for (int64_t t0 = t0_first; t0 < p.tiles && ok; t0 += gridDim.x) {
      const int64_t grow = (t0 + crank) * 128 + 32 * e + lane;
      for (int g = 0; g < nseg; ++g, ++seg) {
        const int ab = (int)(seg % C::NACC);
        if (!warp_wait(&accf[ab], (uint32_t)((seg / C::NACC) & 1), abort, p.status)) {
          ok = false;
          break;
        }
        ptx::tc_fence_after();
        const bool first = g == 0, last = g == nseg - 1;
        const uint32_t abase = tmem + lane_base + (uint32_t)(ab * C::NPAD);
        const uint32_t sbase = tmem + lane_base + C::S_COL;
        // The warp's whole share of the segment comes into registers at once
        // (one wait), and the accumulator goes back to the tensor core before
        // S is touched: S is updated while the next segment accumulates.
        const int col0 = ehalf * C::WCOLS;
        uint32_t a[C::NCH][32];
#pragma unroll
        for (int c = 0; c < C::NCH; ++c) ptx::tmem_ld32_nowait(abase + (uint32_t)(col0 + 32 * c), a[c]);
        ptx::tmem_wait_ld(a[0]);
#pragma unroll
        for (int c = 1; c < C::NCH; ++c) ptx::tmem_regs_ready(a[c]);
        ptx::tc_fence_before();
        __syncwarp();
        if (lane == 0) ptx::mbar_arrive(&acce[ab]);
        // S (+)= A / t in place in a[], 16 columns at a time; the stores of S
        // run from a[], which nothing overwrites before the next segment
#pragma unroll
        for (int c = 0; c < C::NCH; ++c) {
#pragma unroll
          for (int hh = 0; hh < 2; ++hh) {
            const int cc = col0 + 32 * c + 16 * hh;
            uint32_t* ah = &a[c][16 * hh];
            if (first) {
#pragma unroll
              for (int q = 0; q < 16; ++q) ah[q] = __float_as_uint(__uint_as_float(ah[q]) * us);
            } else {
              uint32_t sv[16];
              ptx::tmem_ld16_nowait(sbase + (uint32_t)cc, sv);
              ptx::tmem_wait_ld(sv);
#pragma unroll
              for (int q = 0; q < 16; ++q)
                ah[q] = __float_as_uint(fmaf(__uint_as_float(ah[q]), us, __uint_as_float(sv[q])));
            }
            if (!last) {
              ptx::tmem_st16_from(sbase + (uint32_t)cc, ah);
            } else if (grow < p.m) {
              float* dst = p.Y + grow * p.k + cc;
#pragma unroll
              for (int q = 0; q < 16; ++q)
                if (cc + q < p.k) yb = max(yb, ah[q] & 0x7fffffffu);
              if (cc + 16 <= p.k && (p.k % 4) == 0) {
#pragma unroll
                for (int q = 0; q < 16; q += 4)
                  *reinterpret_cast<float4*>(dst + q) = make_float4(__uint_as_float(ah[q]), __uint_as_float(ah[q + 1]),
                                                                    __uint_as_float(ah[q + 2]), __uint_as_float(ah[q + 3]));
              } else {
#pragma unroll
                for (int q = 0; q < 16; ++q)
                  if (cc + q < p.k) dst[q] = __uint_as_float(ah[q]);
              }
            }
          }
        }
        // S stores land before a[] is reloaded (and before the next fold reads S)
        ptx::tmem_wait_st();
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) yb = max(yb, __shfl_xor_sync(0xffffffffu, yb, o));
    if (lane == 0) {
      if (yb >= 0x7f800000u) {
        if (p.check_y) atomicOr(p.status, ST_NONFINITE);
      } else if (p.ymax) {
        atomic_max_nonneg(p.ymax, __uint_as_float(yb));
      }
    }
  }
  ptx::tc_fence_before();
  __syncthreads();
  // neither CTA leaves while the other may still multicast into it or arrive
  // on its barriers
  ptx::cluster_sync();
  if (warp == C::MMA_W) {
    ptx::tc_fence_after();
    ptx::tmem_dealloc(tmem, C::TMEM_COLS);
  }
}

template <bool E4M3, int NT, bool EXACT_V>
bool launch_cfg(Launcher& L, const CUtensorMap& tm, const Params& p) {
  using C = Cfg<E4M3, NT, EXACT_V>;
  if (cudaFuncSetAttribute(xproj_kernel<E4M3, NT, EXACT_V>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)C::SMEM) != cudaSuccess)
    return false;
  // CTA pairs (clusters of two): an even grid of at most the pairs that can
  // be resident at once (a GPC with an odd number of free SMs leaves one out)
  static int resident = -1;
  if (resident < 0) {
    cudaLaunchConfig_t lc = {};
    lc.gridDim = dim3((unsigned)(L.num_sms / 2 * 2));
    lc.blockDim = dim3(C::THREADS);
    lc.dynamicSmemBytes = C::SMEM;
    int nc = 0;
    if (cudaOccupancyMaxActiveClusters(&nc, xproj_kernel<E4M3, NT, EXACT_V>, &lc) != cudaSuccess || nc < 1) {
      cudaGetLastError();
      nc = L.num_sms / 2;
    }
    resident = nc < L.num_sms / 2 ? nc : L.num_sms / 2;
  }
  const int64_t pairs = (p.tiles + 1) / 2;
  int grid = (int)(pairs < resident ? pairs : resident) * 2;
  if (grid < 2) grid = 2;
  xproj_kernel<E4M3, NT, EXACT_V><<<grid, C::THREADS, C::SMEM, L.stream>>>(tm, p);
  L.count(1);
  return true;
}

template <bool E4M3, bool EXACT_V>
bool launch_nt(Launcher& L, int nt, const CUtensorMap& tm, const Params& p) {
  switch (nt) {
    case 1: return launch_cfg<E4M3, 1, EXACT_V>(L, tm, p);
    case 2: return launch_cfg<E4M3, 2, EXACT_V>(L, tm, p);
    case 3: return launch_cfg<E4M3, 3, EXACT_V>(L, tm, p);
    default: return launch_cfg<E4M3, 4, EXACT_V>(L, tm, p);
  }
}

}  // namespace xp

bool tc_xproj_ok(const void* X, int xt, int64_t ldx, bool exact_v) {
  if (xt == LSPCA_BF16) return ((uintptr_t)X % 16) == 0 && (ldx * 2) % 16 == 0;
  if (xt == LSPCA_E4M3) return !exact_v && ((uintptr_t)X % 16) == 0 && ldx % 16 == 0;
  return false;
}

bool tc_xproj(Launcher& L, const void* X, int xt, int64_t m, int64_t n, int64_t ldx, const void* vtiles,
              const float* vscale, int k, bool exact_v, float* Y, int* status, float* ymax, bool check_y) {
  if (m < 1 || n < 1 || k < 1 || k > 256 || !tc_xproj_ok(X, xt, ldx, exact_v)) return false;
  const bool e4 = xt == LSPCA_E4M3;
  CUtensorMap tm;
  if (e4) {
    if (!make_tmap_2d_sw128(&tm, X, CU_TENSOR_MAP_DATA_TYPE_UINT8, 1, (uint64_t)m, (uint64_t)n, (uint64_t)ldx, 128,
                            128))
      return false;
  } else if (!make_tmap_2d_sw128(&tm, X, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, (uint64_t)m, (uint64_t)n,
                                 (uint64_t)ldx * 2, 128, xp::BK)) {
    return false;
  }
  xp::Params p{};
  p.m = m;
  p.n = n;
  p.k = k;
  p.tiles = (m + 127) / 128;
  p.nks = (int)((n + xp::BK - 1) / xp::BK);
  p.vt = (const uint8_t*)vtiles;
  p.vscale = e4 ? vscale : nullptr;
  p.Y = Y;
  p.ymax = ymax;
  p.check_y = check_y ? 1 : 0;
  p.status = status;
  const int nt = (k + 63) / 64;
  if (e4) return xp::launch_nt<true, false>(L, nt, tm, p);
  return exact_v ? xp::launch_nt<false, true>(L, nt, tm, p) : xp::launch_nt<false, false>(L, nt, tm, p);
}

}  // namespace lspca
