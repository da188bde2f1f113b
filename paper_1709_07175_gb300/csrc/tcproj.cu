// Tensor-core reduction map Y = X V (Sec. III-B.2: pi(x) = V^T x for every
// row) on sm_103a with tcgen05/TMEM.  With V = a dense Omega the same kernel
// computes the sketch U = X Omega (Eq. 1).
//
// GEMM view: M = 128 rows of X per tile, N = k padded to a multiple of 64,
// K = n.  A = the X tile (K-major: rows of X are contiguous in K), B = V
// (MN-major: rows of V are contiguous in N).
//
// Number formats.
// * FP32 X: x s_r = hi + lo with FP16 pieces, where s_r is a power of two
//   chosen per row and per k-step from the row's max |x| in that step (a
//   half-warp reduction over the 64 values the converters already hold), so no
//   extra pass over X is needed; V t = hi + lo likewise with one power of two
//   t from max|V|.  Three products hi*hi + hi*lo + lo*hi.
// * BF16 X: X exact; V split into a BF16 pair; two products.
// * E4M3 X: values widened exactly to BF16; V split as for BF16.
// * V exact in its hi piece (the very sparse Omega: entries 0 and +-1): the
//   products with V's lo piece, which is zero, are skipped and only the hi
//   tiles are copied.  FP32 X is then split into three BF16 pieces
//   x = x0 + x1 + x2 (exact: each piece keeps the top 8 bits of an exactly
//   computed remainder) with no scale, three products, each exact.
//
// Accumulation.  FP32 accumulation of tcgen05.mma into TMEM behaves like
// round-toward-zero on GB300, so the tensor core accumulates short segments
// into a TMEM accumulator A: one k-step (64 columns) for the FP16 pairs, whose
// per-row scales change every k-step, SEG k-steps otherwise.  The epilogue unscales
// each row of a segment by 1 / (s_r t) and folds it into a round-to-nearest
// FP32 running sum S in TMEM, then writes S as the rows of Y after the last
// k-step.  For k <= 128 the accumulator is double-buffered, so the tensor
// core fills one buffer while the epilogue folds the other.
//
// Structure (one persistent CTA per SM):
//   warps 0..CW-1    converters (16 for FP32 X, else 8): 16-byte loads of the X
//                    rows of a k-step, one k-step ahead in two register
//                    buffers in ping-pong, converted into the 128-byte-swizzled
//                    K-major A layout;
//   warps CW..CW+3   epilogue: one per TMEM lane quarter;
//   warp  CW+4       TMEM allocation and the thread that issues tcgen05.mma;
//   warp  CW+5       producer: one cp.async.bulk of the pre-split,
//                    pre-swizzled V tile of each stage.
// All waits are bounded (2 s of %globaltimer): on expiry the kernel records
// ST_TIMEOUT, stops issuing work, waits (bounded) for its copies and MMAs in
// flight and frees TMEM.
#include <type_traits>

#include "common.cuh"
#include "tc.h"
#include "tc_ptx.cuh"

namespace lspca {
namespace tcp {

constexpr int BK = 64;
constexpr int kPrefetchSteps = 2;  // L2 prefetch distance of the converters, in k-steps
constexpr uint64_t kWaitNs = 2000000000ull;
constexpr uint64_t kDrainNs = 100000000ull;

enum XKind { XK_F32 = 0, XK_BF16 = 1, XK_E4M3 = 2 };

struct Params {
  const void* X;
  int64_t ldx;
  int64_t m, n;
  int k;
  const uint8_t* vt;    // pre-tiled V: per k-step [hi | lo], 256 * NPAD bytes
  const float* vscale;  // device: t (FP32 path) at [0]
  float* Y;             // m x k FP32
  int* status;
  const TcProjUnit* units;  // table mode (serving batches): tiles of many requests
  const int* nunits;        // device count of the table
  float* xmax;              // nullable: max|X| out (NaN / Inf in X set ST_NONFINITE instead)
  float* ymax;              // nullable: max|Y| out
};

// The tile being processed: from the single matrix, or from the table.
struct TileInfo {
  const void* X;
  int64_t ldx, m, row0, n;
  int k;
  const uint8_t* vt;
  const float* vscale;
  float* Y;
};

__device__ __forceinline__ TileInfo tile_info(const Params& p, int64_t t) {
  TileInfo ti;
  if (p.units) {
    const TcProjUnit& u = p.units[t];
    ti.X = u.X;
    ti.ldx = u.ldx;
    ti.m = u.m;
    ti.row0 = u.row0;
    ti.n = u.n;
    ti.k = u.k;
    ti.vt = u.vt;
    ti.vscale = u.vscale;
    ti.Y = u.Y;
  } else {
    ti.X = p.X;
    ti.ldx = p.ldx;
    ti.m = p.m;
    ti.row0 = t * 128;
    ti.n = p.n;
    ti.k = p.k;
    ti.vt = p.vt;
    ti.vscale = p.vscale;
    ti.Y = p.Y;
  }
  return ti;
}

template <int XK, int NT, bool EXACT_V>
struct Cfg {
  static constexpr int NPAD = 64 * NT;
  static constexpr bool F32 = XK == XK_F32;
  // FP32 X against an exact V: X as three BF16 pieces x0 + x1 + x2 (exactly
  // x), no scale; FP32 X otherwise: FP16 pair of x s_r with per-row scales
  static constexpr bool SPL3 = F32 && EXACT_V;
  static constexpr bool F16 = F32 && !EXACT_V;          // FP16 operands (else BF16)
  static constexpr int PA = SPL3 ? 3 : (F32 ? 2 : 1);   // A parts
  static constexpr int PB = EXACT_V ? 1 : 2;            // B parts used
  static constexpr uint32_t A_BYTES = 128 * BK * 2;     // 16 KB
  static constexpr uint32_t B_BYTES = BK * NPAD * 2;    // one part
  static constexpr uint32_t SBO_B = NT * 1024;
  static constexpr uint32_t STAGE_BYTES = PB * B_BYTES + PA * A_BYTES;  // [B parts | A parts]
  static constexpr int STAGES = STAGE_BYTES * 4 <= 200 * 1024 ? 4 : STAGE_BYTES * 3 <= 200 * 1024 ? 3 : 2;
  static constexpr int CW = F32 ? 16 : 8;               // converter warps
  static constexpr int CT = CW * 32;
  static constexpr int ES = F32 ? 4 : (XK == XK_BF16 ? 2 : 1);
  static constexpr int EPV = 16 / ES;                   // elements per 16-byte load
  static constexpr int VPR = BK / EPV;                  // 16-byte loads per row of a k-step
  static constexpr int NV = 128 * VPR / CT;             // 16-byte loads per converter thread per k-step
  static constexpr int EW_N = 4;                        // epilogue warps (one per TMEM lane quarter)
  static constexpr int EPI0 = CW;                       // a multiple of 4 (TMEM lane quarters)
  static constexpr int MMA_W = CW + EW_N;
  static constexpr int PROD_W = CW + EW_N + 1;
  static constexpr int THREADS = (CW + EW_N + 2) * 32;
  static constexpr int NACC = NPAD <= 128 ? 2 : 1;      // segment accumulators in TMEM
  static constexpr uint32_t S_COL = NACC * NPAD;        // running sum S after them
  static constexpr int SEG = F16 ? 1 : 8;               // k-steps per accumulation segment
  static constexpr int RING = STAGES + NACC + 1;        // per-row scale slots (FP32 X)
  static constexpr size_t SMEM = 1024 + STAGES * STAGE_BYTES + RING * 128 * 4 + 256 + 8192;
  static_assert(S_COL + NPAD <= 512, "TMEM budget");
  static_assert(NV * CT == 128 * VPR, "converter split");
};

__device__ __forceinline__ float pow2_scale_row(float amax) {
  if (!(amax > 0.f) || !isfinite(amax)) return 1.f;
  int e;
  frexpf(amax, &e);
  return ldexpf(1.f, 14 - e);
}

// The power of two 2^(14 - E), E the exponent with amax < 2^E, from the bits
// of amax (sign cleared): |x| 2^(14 - E) < 2^14 for |x| <= amax.  1 for amax 0
// or non-finite; clamped to 2^127 for subnormal amax.
__device__ __forceinline__ float pow2_scale_bits(uint32_t ab) {
  if (ab == 0u || ab >= 0x7f800000u) return 1.f;
  const int se = min(max(267 - (int)(ab >> 23), 1), 254);  // biased exponent of the scale
  return __uint_as_float((uint32_t)se << 23);
}

// (a, b) -> three BF16 pieces each, v = p0 + p1 + p2 exactly: p0 keeps the top
// 8 significand bits of v (truncation), p1 the top 8 of the exact remainder and
// p2 the last at most 8 bits, so every piece is a BF16 without rounding.  The
// remainders stay normal FP32 numbers (and the pieces exact) for |v| >= 2^-100.
__device__ __forceinline__ void split_b3(float a, float b, uint32_t& p0, uint32_t& p1, uint32_t& p2) {
  const uint32_t a0 = __float_as_uint(a) & 0xffff0000u, b0 = __float_as_uint(b) & 0xffff0000u;
  const float ra = a - __uint_as_float(a0), rb = b - __uint_as_float(b0);
  const uint32_t a1 = __float_as_uint(ra) & 0xffff0000u, b1 = __float_as_uint(rb) & 0xffff0000u;
  const float sa = ra - __uint_as_float(a1), sb = rb - __uint_as_float(b1);
  p0 = __byte_perm(a0, b0, 0x7632);
  p1 = __byte_perm(a1, b1, 0x7632);
  p2 = __byte_perm(__float_as_uint(sa), __float_as_uint(sb), 0x7632);
}

// (a, b) -> FP16 pairs: hi = fp16(v), lo = fp16(v - hi), two of each packed.
__device__ __forceinline__ void split_h2(float a, float b, uint32_t& hi, uint32_t& lo) {
  const __half2 h = __floats2half2_rn(a, b);
  const float2 f = __half22float2(h);
  const __half2 l = __floats2half2_rn(a - f.x, b - f.y);
  hi = *reinterpret_cast<const uint32_t*>(&h);
  lo = *reinterpret_cast<const uint32_t*>(&l);
}

template <int XK, int NT, bool EXACT_V>
__global__ void __launch_bounds__(Cfg<XK, NT, EXACT_V>::THREADS, 1) project_kernel(Params p) {
  using C = Cfg<XK, NT, EXACT_V>;
  constexpr int STAGES = C::STAGES;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  float* scales = reinterpret_cast<float*>(smem + STAGES * C::STAGE_BYTES);
  uint64_t* full = reinterpret_cast<uint64_t*>(scales + C::RING * 128);
  uint64_t* empty = full + STAGES;
  uint64_t* accf = empty + STAGES;  // [NACC]
  uint64_t* acce = accf + C::NACC;  // [NACC]
  uint64_t* drain = acce + C::NACC;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(drain + 1);
  int* abort_flag = reinterpret_cast<int*>(tmem_slot + 1);

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int64_t tiles = p.units ? (int64_t)*p.nunits : (p.m + 127) / 128;

  if (tid == 0) {
    for (int s = 0; s < STAGES; ++s) {
      ptx::mbar_init(&full[s], C::CW + 1);  // converter warps + the producer's expect-tx arrival
      ptx::mbar_init(&empty[s], 1);
    }
    for (int b = 0; b < C::NACC; ++b) {
      ptx::mbar_init(&accf[b], 1);
      ptx::mbar_init(&acce[b], C::EW_N);
    }
    ptx::mbar_init(drain, 1);
    *abort_flag = 0;
    ptx::fence_mbar_init();
  }
  if (warp == C::MMA_W) ptx::tmem_alloc(tmem_slot, 512);
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
  auto ksteps = [&](const TileInfo& ti) { return (int)((ti.n + BK - 1) / BK); };

  if (warp == C::PROD_W) {
    // ------------------------------------------------------------ producer
    if (lane == 0) {
      int64_t step = 0;
      bool ok = true;
      for (int64_t tile = blockIdx.x; tile < tiles && ok; tile += gridDim.x) {
        const TileInfo ti = tile_info(p, tile);
        const int nks = ksteps(ti);
        for (int ks = 0; ks < nks; ++ks, ++step) {
          const int s = (int)(step % STAGES);
          const uint32_t ph = (uint32_t)((step / STAGES) & 1);
          if (!ptx::mbar_wait(&empty[s], ph ^ 1u, kWaitNs)) {
            fail();
            ok = false;
            break;
          }
          if (aborted()) {
            ok = false;
            break;
          }
          ptx::mbar_arrive_expect_tx(&full[s], C::PB * C::B_BYTES);
          ptx::bulk_g2s(sbase + s * C::STAGE_BYTES, ti.vt + (size_t)ks * 2 * C::B_BYTES, C::PB * C::B_BYTES,
                        &full[s]);
        }
      }
      // bounded wait for the copies of the last stages (complete on the
      // normal path, possibly in flight after an abort)
      for (int64_t w = step - 1; w >= 0 && w >= step - STAGES; --w)
        ptx::mbar_wait(&full[w % STAGES], (uint32_t)((w / STAGES) & 1), kDrainNs);
    }
    __syncwarp();
  } else if (warp < C::CW) {
    // ------------------------------------------------------------ converters
    // Thread tid covers, in every k-step, the EPV elements at column cw of the
    // rows r0 + RSTEP q (q < NV) of the tile; those rows' swizzled offsets
    // differ by whole 1024-byte atoms.
    constexpr int RSTEP = C::CT / C::VPR;
    static_assert(RSTEP % 8 == 0, "a thread's rows are whole swizzle atoms apart");
    constexpr uint32_t QOFF = (RSTEP / 8) * 1024u;
    const int r0 = tid / C::VPR, cw = (tid % C::VPR) * C::EPV;
    const uint32_t soff = ptx::k_sw128_offset(r0, cw);
    // Load cursor: tile lt, its k-step lk of lnk; lp = the address of (row r0,
    // column cw) of k-step lk; lrows = rows of the tile that exist.
    int64_t lt = blockIdx.x, lrs = 0, ln = 0;
    int lk = 0, lnk = 0, lrows = 0;
    const uint8_t* lp = nullptr;
    auto enter = [&]() {
      lk = 0;
      if (lt >= tiles) return;
      const TileInfo ti = tile_info(p, lt);
      lnk = ksteps(ti);
      ln = ti.n;
      lrows = (int)min(ti.m - ti.row0, (int64_t)128);
      const int64_t rb = ti.ldx * C::ES;
      lrs = rb * RSTEP;
      lp = (const uint8_t*)ti.X + (ti.row0 + r0) * rb + cw * C::ES;
    };
    // loads of the cursor's k-step; vc = its columns that exist (BK: all)
    auto issue = [&](uint4 (&dst)[C::NV], int& vc) {
      const int64_t left = ln - (int64_t)lk * BK;
      vc = left >= BK ? BK : (int)left;
      if (lrows == 128 && vc == BK) {
#pragma unroll
        for (int q = 0; q < C::NV; ++q)
          asm volatile("ld.global.nc.L1::no_allocate.v4.u32 {%0, %1, %2, %3}, [%4];"
                       : "=r"(dst[q].x), "=r"(dst[q].y), "=r"(dst[q].z), "=r"(dst[q].w)
                       : "l"(lp + q * lrs));
      } else {
#pragma unroll
        for (int q = 0; q < C::NV; ++q) {
          if (r0 + RSTEP * q < lrows && cw < vc) {
            asm volatile("ld.global.nc.L1::no_allocate.v4.u32 {%0, %1, %2, %3}, [%4];"
                         : "=r"(dst[q].x), "=r"(dst[q].y), "=r"(dst[q].z), "=r"(dst[q].w)
                         : "l"(lp + q * lrs));
          } else {
            dst[q] = make_uint4(0u, 0u, 0u, 0u);
          }
        }
      }
      // L2 prefetch of this thread's rows two k-steps ahead (one per 128-byte
      // line; within the tile's rows, and short of a partial last k-step)
      if (lk + kPrefetchSteps < lnk - (int)((ln & (BK - 1)) != 0) && ((cw * C::ES) & 127) == 0) {
#pragma unroll
        for (int q = 0; q < C::NV; ++q)
          if (r0 + RSTEP * q < lrows) ptx::prefetch_l2(lp + kPrefetchSteps * BK * C::ES + q * lrs);
      }
      lp += BK * C::ES;
      if (++lk >= lnk) {
        lt += gridDim.x;
        enter();
      }
    };
    uint32_t xb = 0u;   // max over the |x| seen, as FP32 bits (>= 0x7f800000: NaN / Inf)
    uint32_t xb2 = 0u;  // three-piece path: max of the BF16 leading pieces' |bits| per half
    auto store = [&](const uint4 (&r)[C::NV], uint32_t st, int slot, int vc) {
      const uint32_t a_hi = st + C::PB * C::B_BYTES, a_lo = a_hi + C::A_BYTES;
      const bool tail = vc < BK;  // the k-step runs past the last column
#pragma unroll
      for (int q = 0; q < C::NV; ++q) {
        const uint32_t off = soff + q * QOFF;
        if constexpr (C::SPL3) {
          float v[4] = {__uint_as_float(r[q].x), __uint_as_float(r[q].y), __uint_as_float(r[q].z),
                        __uint_as_float(r[q].w)};
          if (tail) {
#pragma unroll
            for (int u = 0; u < 4; ++u)
              if (cw + u >= vc) v[u] = 0.f;
          }
          uint32_t p0[2], p1[2], p2[2];
          split_b3(v[0], v[1], p0[0], p1[0], p2[0]);
          split_b3(v[2], v[3], p0[1], p1[1], p2[1]);
          // the leading piece keeps x's sign, exponent and top 7 fraction
          // bits: its max is max|x| rounded toward zero, and NaN / Inf stay
          // >= 0x7f80
          xb2 = __vmaxu2(xb2, __vmaxu2(p0[0] & 0x7fff7fffu, p0[1] & 0x7fff7fffu));
          asm volatile("st.shared.v2.b32 [%0], {%1, %2};" ::"r"(a_hi + off), "r"(p0[0]), "r"(p0[1]) : "memory");
          asm volatile("st.shared.v2.b32 [%0], {%1, %2};" ::"r"(a_lo + off), "r"(p1[0]), "r"(p1[1]) : "memory");
          asm volatile("st.shared.v2.b32 [%0], {%1, %2};" ::"r"(a_lo + C::A_BYTES + off), "r"(p2[0]), "r"(p2[1])
                       : "memory");
        } else if constexpr (XK == XK_F32) {
          float v[4] = {__uint_as_float(r[q].x), __uint_as_float(r[q].y), __uint_as_float(r[q].z),
                        __uint_as_float(r[q].w)};
          if (tail) {
#pragma unroll
            for (int u = 0; u < 4; ++u)
              if (cw + u >= vc) v[u] = 0.f;
          }
          uint32_t mb = __vimax3_u32(__float_as_uint(v[0]) & 0x7fffffffu, __float_as_uint(v[1]) & 0x7fffffffu,
                                     max(__float_as_uint(v[2]) & 0x7fffffffu, __float_as_uint(v[3]) & 0x7fffffffu));
          xb = max(xb, mb);
          // the row's 16 loads sit in one half-warp: max over that half
          static_assert(C::VPR == 16, "one row per half-warp");
          mb = __reduce_max_sync(lane < 16 ? 0x0000ffffu : 0xffff0000u, mb);
          const float sc = pow2_scale_bits(mb);
          if (cw == 0) scales[slot * 128 + r0 + RSTEP * q] = sc;  // FP16 path only
          uint32_t h0, l0, h1, l1;
          split_h2(v[0] * sc, v[1] * sc, h0, l0);
          split_h2(v[2] * sc, v[3] * sc, h1, l1);
          asm volatile("st.shared.v2.b32 [%0], {%1, %2};" ::"r"(a_hi + off), "r"(h0), "r"(h1) : "memory");
          asm volatile("st.shared.v2.b32 [%0], {%1, %2};" ::"r"(a_lo + off), "r"(l0), "r"(l1) : "memory");
        } else if constexpr (XK == XK_BF16) {
          uint4 v = r[q];
          if (tail && cw + 8 > vc) {
            uint16_t* e = reinterpret_cast<uint16_t*>(&v);
#pragma unroll
            for (int u = 0; u < 8; ++u)
              if (cw + u >= vc) e[u] = 0;
          }
          xb2 = __vmaxu2(xb2, __vmaxu2(__vmaxu2(v.x & 0x7fff7fffu, v.y & 0x7fff7fffu),
                                       __vmaxu2(v.z & 0x7fff7fffu, v.w & 0x7fff7fffu)));
          asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(a_hi + off), "r"(v.x), "r"(v.y), "r"(v.z),
                       "r"(v.w)
                       : "memory");
        } else {
          const __nv_fp8_e4m3* e8 = reinterpret_cast<const __nv_fp8_e4m3*>(&r[q]);
          uint32_t w[8];
#pragma unroll
          for (int u = 0; u < 8; ++u) {
            const float a = (!tail || cw + 2 * u < vc) ? float(e8[2 * u]) : 0.f;
            const float b = (!tail || cw + 2 * u + 1 < vc) ? float(e8[2 * u + 1]) : 0.f;
            xb = max(xb, max(__float_as_uint(a) & 0x7fffffffu, __float_as_uint(b) & 0x7fffffffu));
            __nv_bfloat162 h2 = __floats2bfloat162_rn(a, b);
            w[u] = *reinterpret_cast<uint32_t*>(&h2);
          }
          // columns cw .. cw + 7 and cw + 8 .. cw + 15: the second half is the
          // next 16-byte chunk of the row (cw is a multiple of 16)
          asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(a_hi + off), "r"(w[0]), "r"(w[1]),
                       "r"(w[2]), "r"(w[3])
                       : "memory");
          asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(a_hi + (off ^ 16u)), "r"(w[4]), "r"(w[5]),
                       "r"(w[6]), "r"(w[7])
                       : "memory");
        }
      }
    };
    // k-steps of this CTA over all its tiles
    int64_t total = 0;
    if (!p.units) {
      const int64_t mine = tiles > blockIdx.x ? (tiles - 1 - blockIdx.x) / gridDim.x + 1 : 0;
      total = mine * ksteps(tile_info(p, 0));
    } else {
      for (int64_t t = blockIdx.x; t < tiles; t += gridDim.x) total += ksteps(tile_info(p, t));
    }
    // Two register buffers in ping-pong: the loads of k-step t + 1 are issued
    // before k-step t is converted and consumed one full iteration later (a
    // register copy out of a prefetch buffer would wait for them at once).
    int64_t step = 0;
    uint32_t s = 0, ph = 0;
    int slot = 0;
    auto body = [&](const uint4 (&cur)[C::NV], int cvc, uint4 (&nxt)[C::NV], int& nvc) -> bool {
      if (step + 1 < total) issue(nxt, nvc);
      if (!ptx::mbar_wait(&empty[s], ph ^ 1u, kWaitNs)) {
        fail();
        return false;
      }
      if (aborted()) return false;
      store(cur, sbase + s * C::STAGE_BYTES, slot, cvc);
      ptx::fence_proxy_async_smem();
      __syncwarp();
      if (lane == 0) ptx::mbar_arrive(&full[s]);
      if (++s == (uint32_t)STAGES) {
        s = 0;
        ph ^= 1u;
      }
      if (++slot == C::RING) slot = 0;
      return ++step < total;
    };
    uint4 ra[C::NV], rb[C::NV];
    int va = 0, vb = 0;
    if (total > 0) {
      enter();
      issue(ra, va);
      while (body(ra, va, rb, vb) && body(rb, vb, ra, va)) {
      }
    }
    xb = max(xb, max(xb2 >> 16, xb2 & 0xffffu) << 16);  // BF16 bits widen to FP32 bits
    if (p.xmax) {
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) xb = max(xb, __shfl_xor_sync(0xffffffffu, xb, o));
      if (lane == 0) {
        if (xb >= 0x7f800000u) atomicOr(p.status, ST_NONFINITE);
        else atomic_max_nonneg(p.xmax, __uint_as_float(xb));
      }
    }
  } else if (warp == C::MMA_W) {
    // ------------------------------------------------------------ MMA issuer
    if (lane == 0) {
      constexpr uint32_t idesc = ptx::idesc_f16(C::F16 ? 0 : 1, 128, C::NPAD, 0, 1);
      int64_t step = 0, seg = 0;
      bool ok = true;
      for (int64_t tile = blockIdx.x; tile < tiles && ok; tile += gridDim.x) {
        const int nks = ksteps(tile_info(p, tile));
        for (int ks = 0; ks < nks && ok; ++ks, ++step) {
          const bool seg_start = (ks % C::SEG) == 0;
          const int ab = (int)(seg % C::NACC);
          if (seg_start) {
            // wait until the epilogue has folded the segment that last used buffer ab
            if (!ptx::mbar_wait(&acce[ab], (uint32_t)(((seg / C::NACC) & 1) ^ 1), kWaitNs)) {
              fail();
              ok = false;
              break;
            }
            ptx::tc_fence_after();
          }
          const int s = (int)(step % STAGES);
          const uint32_t ph = (uint32_t)((step / STAGES) & 1);
          if (!ptx::mbar_wait(&full[s], ph, kWaitNs) || aborted()) {
            if (!aborted()) fail();
            ok = false;
            break;
          }
          ptx::tc_fence_after();
          const uint32_t st = sbase + s * C::STAGE_BYTES;
          const uint32_t b_hi = st, a_hi = st + C::PB * C::B_BYTES;
          const uint32_t d = tmem + (uint32_t)(ab * C::NPAD);
          // descriptors of the stage's operands; K slices and pieces are offsets
          const uint64_t adh0 = ptx::desc_sw128(a_hi, 16, 1024);
          const uint64_t bdh0 = ptx::desc_sw128(b_hi, 1024, C::SBO_B);
#pragma unroll
          for (int kk = 0; kk < BK / 16; ++kk) {
            const uint64_t adh = ptx::desc_advance(adh0, kk * 32);
            const uint64_t bdh = ptx::desc_advance(bdh0, kk * 2 * C::SBO_B);
            ptx::mma_f16(d, adh, bdh, idesc, (seg_start && kk == 0) ? 0u : 1u);
            if (!EXACT_V) ptx::mma_f16(d, adh, ptx::desc_advance(bdh, C::B_BYTES), idesc, 1u);
            if (C::PA >= 2) ptx::mma_f16(d, ptx::desc_advance(adh, C::A_BYTES), bdh, idesc, 1u);
            if (C::PA == 3) ptx::mma_f16(d, ptx::desc_advance(adh, 2 * C::A_BYTES), bdh, idesc, 1u);
          }
          ptx::mma_commit(&empty[s]);
          if ((ks % C::SEG) == C::SEG - 1 || ks == nks - 1) {
            ptx::mma_commit(&accf[ab]);
            ++seg;
          }
        }
      }
      ptx::mma_commit(drain);
      if (!ptx::mbar_wait(drain, 0u, kWaitNs)) atomicOr(p.status, ST_TIMEOUT);
    }
    __syncwarp();
  } else {
    // ------------------------------------------------------------ epilogue
    const int e = (warp - C::EPI0) & 3;       // TMEM lane quarter
    const int ehalf = (warp - C::EPI0) >> 2;  // which share of the columns this warp folds
    const uint32_t lane_base = (uint32_t)(32 * e) << 16;
    constexpr int EW = 16;  // TMEM columns per fold chunk
    uint32_t yb = 0u;       // max|Y| written, as FP32 bits
    int64_t step = 0, seg = 0;
    bool ok = true;
    for (int64_t tile = blockIdx.x; tile < tiles && ok; tile += gridDim.x) {
      const TileInfo ti = tile_info(p, tile);
      const float inv_t = C::F16 ? 1.f / *ti.vscale : 1.f;
      const int nks = ksteps(ti);
      const int nseg = (nks + C::SEG - 1) / C::SEG;
      const int row = 32 * e + lane;
      const int64_t grow = ti.row0 + row;
      for (int g = 0; g < nseg; ++g, ++seg) {
        const int ab = (int)(seg % C::NACC);
        if (!ptx::mbar_wait(&accf[ab], (uint32_t)((seg / C::NACC) & 1), kWaitNs) || aborted()) {
          if (!aborted()) fail();
          ok = false;
          break;
        }
        ptx::tc_fence_after();
        // FP32 X: one k-step per segment, unscaled by its per-row scale
        const float us = C::F16 ? inv_t / scales[(int)(step % C::RING) * 128 + row] : 1.f;
        const bool first = g == 0, last = g == nseg - 1;
        const uint32_t abase = tmem + lane_base + (uint32_t)(ab * C::NPAD);
        const uint32_t sbase_t = tmem + lane_base + C::S_COL;
#pragma unroll 1
        constexpr int WCOLS = C::NPAD * 4 / C::EW_N;  // columns folded by one epilogue warp
        for (int cc = ehalf * WCOLS; cc < (ehalf + 1) * WCOLS; cc += EW) {
          uint32_t a[EW], r[EW];
          // the previous chunk's store of S has to land before r is reloaded
          ptx::tmem_wait_st(r);
          ptx::tmem_ld16_nowait(abase + (uint32_t)cc, a);
          if (!first) ptx::tmem_ld16_nowait(sbase_t + (uint32_t)cc, r);
          ptx::tmem_wait_ld(a);
          if (first) {
#pragma unroll
            for (int q = 0; q < EW; ++q) r[q] = __float_as_uint(__uint_as_float(a[q]) * us);
          } else {
            ptx::tmem_regs_ready(r);
#pragma unroll
            for (int q = 0; q < EW; ++q)
              r[q] = __float_as_uint(fmaf(__uint_as_float(a[q]), us, __uint_as_float(r[q])));
          }
          if (!last) {
            ptx::tmem_st16_nowait(sbase_t + (uint32_t)cc, r);
          } else if (grow < ti.m) {
            float* dst = ti.Y + grow * ti.k + cc;
#pragma unroll
            for (int q = 0; q < EW; ++q)
              if (cc + q < ti.k) yb = max(yb, r[q] & 0x7fffffffu);
            if (cc + EW <= ti.k && (ti.k % 4) == 0) {
#pragma unroll
              for (int q = 0; q < EW; q += 4)
                *reinterpret_cast<float4*>(dst + q) = make_float4(__uint_as_float(r[q]), __uint_as_float(r[q + 1]),
                                                                  __uint_as_float(r[q + 2]),
                                                                  __uint_as_float(r[q + 3]));
            } else {
#pragma unroll
              for (int q = 0; q < EW; ++q)
                if (cc + q < ti.k) dst[q] = __uint_as_float(r[q]);
            }
          }
        }
        ptx::tc_fence_before();
        __syncwarp();
        if (lane == 0) ptx::mbar_arrive(&acce[ab]);
        step += (g == nseg - 1) ? nks - g * C::SEG : C::SEG;
      }
    }
    ptx::tmem_wait_st();
    if (p.ymax) {
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) yb = max(yb, __shfl_xor_sync(0xffffffffu, yb, o));
      if (lane == 0 && yb < 0x7f800000u) atomic_max_nonneg(p.ymax, __uint_as_float(yb));
    }
  }
  __syncthreads();
  if (warp == C::MMA_W) {
    ptx::tc_fence_after();
    ptx::tmem_dealloc(tmem, 512);
  }
}

// V (n x k FP32) -> per k-step tiles [hi | lo] in the MN-major SW128 layout
// (8 K-rows x 64 N-columns per 1024-byte atom, N-atoms adjacent), zero padded
// to NPAD columns and to whole k-steps.  FP32 path: FP16 pair of V * t with t
// a power of two from max|V| (vscale[0] = t); else a BF16 pair of V.
__global__ void tile_v_kernel(const float* __restrict__ V, int64_t n, int k, int npad, int f16, const float* amax,
                              float* vscale, uint8_t* __restrict__ out) {
  const int nt = npad / 64;
  const int nks = (int)((n + BK - 1) / BK);
  const uint32_t sbo = nt * 1024;
  const size_t part = (size_t)BK * npad * 2;
  float t = 1.f;
  if (f16) {
    t = pow2_scale_row(*amax);
    if (blockIdx.x == 0 && threadIdx.x == 0) *vscale = t;
  }
  const int64_t total = (int64_t)nks * BK * npad;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int c = (int)(e % npad);
    const int64_t j = e / npad;  // global row of V
    const int ks = (int)(j / BK), kr = (int)(j % BK);
    const float v = (j < n && c < k) ? V[j * k + c] : 0.f;
    uint16_t hb, lb;
    if (f16) {
      const __half h = __float2half_rn(v * t);
      const __half l = __float2half_rn(v * t - __half2float(h));
      hb = *reinterpret_cast<const uint16_t*>(&h);
      lb = *reinterpret_cast<const uint16_t*>(&l);
    } else {
      const __nv_bfloat16 h = __float2bfloat16_rn(v);
      const __nv_bfloat16 l = __float2bfloat16_rn(v - __bfloat162float(h));
      hb = *reinterpret_cast<const uint16_t*>(&h);
      lb = *reinterpret_cast<const uint16_t*>(&l);
    }
    uint8_t* base = out + (size_t)ks * 2 * part;
    const uint32_t off = ptx::mn_sw128_offset(kr, c, sbo);
    *reinterpret_cast<uint16_t*>(base + off) = hb;
    *reinterpret_cast<uint16_t*>(base + part + off) = lb;
  }
}

// ---------------------------------------------------------------------------
// Y = X V for FP32 X and k <= 128 with the A operand in tensor memory: the
// sketch U = X Omega against the very sparse Omega (PV = 1: Omega is exact in
// one BF16 piece) and the reduction map Y = X V (PV = 3: V split exactly into
// three BF16 pieces v = v0 + v1 + v2 by tile_v3_kernel).
//
// X is split into three exact BF16 pieces x = x0 + x1 + x2 as in
// project_kernel's three-piece path.  PV = 1 takes the three products x_a v0;
// PV = 3 takes the six products x_a v_b with a + b <= 2 (the three left out are
// below 2^-24 |x| |v| together, under FP32 rounding of the product).  Every
// product is exact; the tensor core accumulates segments of SEG k-steps,
// folded into a round-to-nearest FP32 sum.  The converter warps write the
// pieces straight into TMEM with tcgen05.st and the MMA reads A from there, so
// the pieces never pass through shared memory: the tensor core's
// shared-memory reads (B only) no longer compete with converter stores.  The
// running sum S moves to shared memory (row-private, padded rows), which frees
// TMEM for a double-buffered accumulator plus the A stages.
//
// Thread mapping: converter warp w owns TMEM lane quarter w % 4 (tile rows
// 32 (w % 4) .. + 31, one row per lane) and the 16 columns 16 (w / 4) .. + 15
// of every 64-column k-step: two 32-byte loads of its row per k-step, one
// 16-column MMA slice (8 TMEM columns) per piece.  A k-step's register buffer
// is freed by the split into pieces and takes the loads of the k-step two
// ahead right after the TMEM stores are issued; an L2 prefetch runs two
// k-steps further.
//
// TMEM columns: [0, NACC NPAD) accumulators; then A_STAGES stages of
// 3 pieces x 32 columns.  Warps: 16 converters, 4 epilogue (one per lane
// quarter), the MMA issuer (also allocates TMEM), a producer (bulk copy of
// each k-step's V tile, PV parts).  Waits are bounded as in project_kernel.
//
// Segments.  The tensor core's FP32 accumulation truncates, so every
// accumulating MMA that changes the sum costs up to an ulp of it.  PV = 1: 16
// k-steps (1,024 columns of X) -- most products of the very sparse Omega are
// zero and leave the sum unchanged; measured on GB300, 16 is 5 % faster than 8
// and stays within the sequential-summation bound of the FP64 sum.  PV = 3: one
// k-step, with the large product last (see prod_pieces): about four
// full-size truncations per fold.
namespace sk {
constexpr int CW = 16, EW_N = 4, EPI0 = 16, MMA_W = 20, PROD_W = 21;
constexpr int THREADS = 22 * 32;
}  // namespace sk

template <int NT, int PV>
struct SkCfg {
  static_assert(PV == 1 || PV == 3, "V pieces");
  static constexpr int NPAD = 64 * NT;
  static constexpr int NACC = 2;  // accumulators in TMEM
  static constexpr int SEG = PV == 1 ? 16 : 1;
  static constexpr int NPROD = PV == 1 ? 3 : 6;
  static constexpr uint32_t B_BYTES = BK * NPAD * 2;           // one part of a k-step's V tile
  static constexpr uint32_t STAGE_B = PV * B_BYTES;             // the parts used
  static constexpr uint32_t TILE_STRIDE = (PV == 1 ? 2 : 3) * B_BYTES;  // bytes per k-step in the tiles
  static constexpr uint32_t SBO_B = NT * 1024;
  static constexpr int B_STAGES = PV == 1 ? 6 : 3;
  static constexpr uint32_t ACOL0 = NACC * NPAD;  // first A column
  static constexpr int A_STAGES = (512 - ACOL0) / 96 < 4 ? (512 - ACOL0) / 96 : 4;
  static constexpr int SST = NPAD + 4;  // floats per row of S (padding spreads the rows over the banks)
  static constexpr size_t SMEM = 1024 + (size_t)B_STAGES * STAGE_B + (size_t)128 * SST * 4 + 512;
  static_assert(ACOL0 + A_STAGES * 96 <= 512, "TMEM budget");
  static_assert(A_STAGES >= 2, "A stages");
  static_assert(SMEM <= 227 * 1024, "shared memory");
};

// Pieces (a, b) of the products x_a v_b, in issue order: for PV = 3 the five
// cross products first, smallest first, while the accumulator is small, and
// x0 v0 last, so that only its four slices truncate at the full size of the
// sum.
__device__ __forceinline__ void prod_pieces(int q, int pv, int& a, int& b) {
  if (pv == 1) {
    a = q;
    b = 0;
  } else {
    constexpr int A6[6] = {2, 1, 0, 1, 0, 0}, B6[6] = {0, 1, 2, 0, 1, 0};
    a = A6[q];
    b = B6[q];
  }
}

template <int NT, int PV>
__global__ void __launch_bounds__(sk::THREADS, 1) tmem_a_kernel(Params p) {
  using C = SkCfg<NT, PV>;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  float* Ssm = reinterpret_cast<float*>(smem + C::B_STAGES * C::STAGE_B);
  uint64_t* fullA = reinterpret_cast<uint64_t*>(Ssm + 128 * C::SST);
  uint64_t* emptyA = fullA + C::A_STAGES;
  uint64_t* fullB = emptyA + C::A_STAGES;
  uint64_t* emptyB = fullB + C::B_STAGES;
  uint64_t* accf = emptyB + C::B_STAGES;  // [NACC]
  uint64_t* acce = accf + C::NACC;        // [NACC]
  uint64_t* drain = acce + C::NACC;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(drain + 1);
  int* abort_flag = reinterpret_cast<int*>(tmem_slot + 1);

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int64_t tiles = (p.m + 127) / 128;
  const int nks = (int)((p.n + BK - 1) / BK);
  if (tid == 0) {
    for (int s = 0; s < C::A_STAGES; ++s) {
      ptx::mbar_init(&fullA[s], sk::CW);
      ptx::mbar_init(&emptyA[s], 1);
    }
    for (int s = 0; s < C::B_STAGES; ++s) {
      ptx::mbar_init(&fullB[s], 1);
      ptx::mbar_init(&emptyB[s], 1);
    }
    for (int b = 0; b < C::NACC; ++b) {
      ptx::mbar_init(&accf[b], 1);
      ptx::mbar_init(&acce[b], sk::EW_N);
    }
    ptx::mbar_init(drain, 1);
    *abort_flag = 0;
    ptx::fence_mbar_init();
  }
  if (warp == sk::MMA_W) ptx::tmem_alloc(tmem_slot, 512);
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
  const int64_t my_tiles = tiles > blockIdx.x ? (tiles - 1 - blockIdx.x) / gridDim.x + 1 : 0;
  const int64_t total = my_tiles * nks;  // k-steps of this CTA

  if (warp == sk::PROD_W) {
    // ------------------------------------------------------------ producer
    if (lane == 0) {
      int64_t step = 0;
      uint32_t s = 0, ph = 0;
      int ks = 0;
      for (; step < total; ++step) {
        if (!ptx::mbar_wait(&emptyB[s], ph ^ 1u, kWaitNs)) {
          fail();
          break;
        }
        if (aborted()) break;
        ptx::mbar_arrive_expect_tx(&fullB[s], C::STAGE_B);
        ptx::bulk_g2s(sbase + s * C::STAGE_B, p.vt + (size_t)ks * C::TILE_STRIDE, C::STAGE_B, &fullB[s]);
        if (++ks == nks) ks = 0;
        if (++s == (uint32_t)C::B_STAGES) {
          s = 0;
          ph ^= 1u;
        }
      }
      // bounded wait for the copies of the last stages issued
      for (int64_t w = step - 1; w >= 0 && w >= step - C::B_STAGES; --w)
        ptx::mbar_wait(&fullB[w % C::B_STAGES], (uint32_t)((w / C::B_STAGES) & 1), kDrainNs);
    }
    __syncwarp();
  } else if (warp < sk::CW) {
    // ------------------------------------------------------------ converters
    const int qd = warp & 3, j = warp >> 2;
    const uint32_t lane_base = (uint32_t)(32 * qd) << 16;
    const int r = 32 * qd + lane;  // row of the tile
    const int64_t rb = p.ldx * 4;  // row bytes
    uint32_t xb2 = 0u;
    // load cursor: tile lt, k-step lk
    int64_t lt = blockIdx.x;
    int lk = 0;
    auto issue = [&](float (&v)[16]) {
      const int64_t row = lt * 128 + r;
      const int64_t c = (int64_t)lk * BK + 16 * j;
      const float* src = reinterpret_cast<const float*>((const uint8_t*)p.X + row * rb) + c;
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        if (row < p.m && c + 8 * h < p.n) {
          asm volatile("ld.global.nc.L1::no_allocate.v8.f32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
                       : "=f"(v[8 * h + 0]), "=f"(v[8 * h + 1]), "=f"(v[8 * h + 2]), "=f"(v[8 * h + 3]),
                         "=f"(v[8 * h + 4]), "=f"(v[8 * h + 5]), "=f"(v[8 * h + 6]), "=f"(v[8 * h + 7])
                       : "l"(src + 8 * h));
          if (c + 8 * h + 8 > p.n) {
#pragma unroll
            for (int u = 0; u < 8; ++u)
              if (c + 8 * h + u >= p.n) v[8 * h + u] = 0.f;
          }
        } else {
#pragma unroll
          for (int u = 0; u < 8; ++u) v[8 * h + u] = 0.f;
        }
      }
      // L2 prefetch of the row's segment two k-steps ahead (one per 128-byte
      // line: the warps with j even start a line)
      if ((j & 1) == 0 && lk + kPrefetchSteps < nks - (int)((p.n & (BK - 1)) != 0) && row < p.m)
        ptx::prefetch_l2(src + kPrefetchSteps * BK);
      if (++lk == nks) {
        lk = 0;
        lt += gridDim.x;
      }
    };
    int64_t step = 0;
    uint32_t s = 0, ph = 0;
    auto body = [&](float (&cur)[16]) -> bool {
      if (!ptx::mbar_wait(&emptyA[s], ph ^ 1u, kWaitNs)) {
        fail();
        return false;
      }
      if (aborted()) return false;
      ptx::tc_fence_after();
      uint32_t p0[8], p1[8], p2[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) split_b3(cur[2 * u], cur[2 * u + 1], p0[u], p1[u], p2[u]);
#pragma unroll
      for (int u = 0; u < 8; u += 2) xb2 = __vmaxu2(xb2, __vmaxu2(p0[u] & 0x7fff7fffu, p0[u + 1] & 0x7fff7fffu));
      const uint32_t ta = tmem + lane_base + C::ACOL0 + s * 96 + 8 * j;
      ptx::tmem_st8(ta, p0);
      ptx::tmem_st8(ta + 32, p1);
      ptx::tmem_st8(ta + 64, p2);
      if (step + 2 < total) issue(cur);
      ptx::tmem_wait_st();
      ptx::tc_fence_before();
      __syncwarp();
      if (lane == 0) ptx::mbar_arrive(&fullA[s]);
      if (++s == (uint32_t)C::A_STAGES) {
        s = 0;
        ph ^= 1u;
      }
      return ++step < total;
    };
    float va[16], vb[16];
    if (total > 0) {
      issue(va);
      if (total > 1) issue(vb);
      while (body(va) && body(vb)) {
      }
    }
    uint32_t xb = max(xb2 >> 16, xb2 & 0xffffu) << 16;  // BF16 bits widen to FP32 bits
    if (p.xmax) {
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) xb = max(xb, __shfl_xor_sync(0xffffffffu, xb, o));
      if (lane == 0) {
        if (xb >= 0x7f800000u) atomicOr(p.status, ST_NONFINITE);
        else atomic_max_nonneg(p.xmax, __uint_as_float(xb));
      }
    }
  } else if (warp == sk::MMA_W) {
    // ------------------------------------------------------------ MMA issuer
    if (lane == 0) {
      constexpr uint32_t idesc = ptx::idesc_f16(1, 128, C::NPAD, 0, 1);
      int64_t step = 0, seg = 0;
      uint32_t sa = 0, pa = 0, sb = 0, pb = 0;
      bool ok = true;
      for (int64_t t = 0; t < my_tiles && ok; ++t) {
        for (int ks = 0; ks < nks && ok; ++ks, ++step) {
          const bool seg_start = (ks % C::SEG) == 0;
          const int ab = (int)(seg % C::NACC);
          if (seg_start) {
            if (!ptx::mbar_wait(&acce[ab], (uint32_t)(((seg / C::NACC) & 1) ^ 1), kWaitNs)) {
              fail();
              ok = false;
              break;
            }
            ptx::tc_fence_after();
          }
          if (!ptx::mbar_wait(&fullB[sb], pb, kWaitNs) || !ptx::mbar_wait(&fullA[sa], pa, kWaitNs) || aborted()) {
            if (!aborted()) fail();
            ok = false;
            break;
          }
          ptx::tc_fence_after();
          const uint32_t d = tmem + (uint32_t)(ab * C::NPAD);
          const uint64_t bd0 = ptx::desc_sw128(sbase + sb * C::STAGE_B, 1024, C::SBO_B);
          const uint32_t a0 = tmem + C::ACOL0 + sa * 96;
#pragma unroll
          for (int q = 0; q < C::NPROD; ++q) {
            int pa, pb;
            prod_pieces(q, PV, pa, pb);
#pragma unroll
            for (int kk = 0; kk < BK / 16; ++kk)
              ptx::mma_f16_ts(d, a0 + pa * 32 + kk * 8,
                              ptx::desc_advance(bd0, kk * 2 * C::SBO_B + pb * C::B_BYTES), idesc,
                              (seg_start && kk == 0 && q == 0) ? 0u : 1u);
          }
          ptx::mma_commit(&emptyA[sa]);
          ptx::mma_commit(&emptyB[sb]);
          if (++sa == (uint32_t)C::A_STAGES) {
            sa = 0;
            pa ^= 1u;
          }
          if (++sb == (uint32_t)C::B_STAGES) {
            sb = 0;
            pb ^= 1u;
          }
          if ((ks % C::SEG) == C::SEG - 1 || ks == nks - 1) {
            ptx::mma_commit(&accf[ab]);
            ++seg;
          }
        }
      }
      ptx::mma_commit(drain);
      if (!ptx::mbar_wait(drain, 0u, kWaitNs)) atomicOr(p.status, ST_TIMEOUT);
    }
    __syncwarp();
  } else {
    // ------------------------------------------------------------ epilogue
    const int e = warp & 3;  // TMEM lane quarter (EPI0 is a multiple of 4)
    const uint32_t lane_base = (uint32_t)(32 * e) << 16;
    const int row = 32 * e + lane;
    float* srow = Ssm + row * C::SST;
    const int nseg = (nks + C::SEG - 1) / C::SEG;
    uint32_t yb = 0u;
    int64_t seg = 0;
    bool ok = true;
    for (int64_t t = 0; t < my_tiles && ok; ++t) {
      const int64_t grow = (blockIdx.x + t * gridDim.x) * 128 + row;
      for (int g = 0; g < nseg; ++g, ++seg) {
        const int ab = (int)(seg % C::NACC);
        if (!ptx::mbar_wait(&accf[ab], (uint32_t)((seg / C::NACC) & 1), kWaitNs) || aborted()) {
          if (!aborted()) fail();
          ok = false;
          break;
        }
        ptx::tc_fence_after();
        const bool first = g == 0, last = g == nseg - 1;
        const uint32_t abase = tmem + lane_base + (uint32_t)(ab * C::NPAD);
#pragma unroll 1
        for (int cc = 0; cc < C::NPAD; cc += 32) {
          uint32_t a[32];
          ptx::tmem_ld32_nowait(abase + (uint32_t)cc, a);
          ptx::tmem_wait_ld(a);
          float* y = reinterpret_cast<float*>(a);  // the sum is formed in place
          if (!first) {
#pragma unroll
            for (int q = 0; q < 32; q += 4) {
              const float4 sv = *reinterpret_cast<const float4*>(srow + cc + q);
              y[q] += sv.x;
              y[q + 1] += sv.y;
              y[q + 2] += sv.z;
              y[q + 3] += sv.w;
            }
          }
          if (!last) {
#pragma unroll
            for (int q = 0; q < 32; q += 4)
              *reinterpret_cast<float4*>(srow + cc + q) = make_float4(y[q], y[q + 1], y[q + 2], y[q + 3]);
          } else if (grow < p.m) {
            float* dst = p.Y + grow * p.k + cc;
#pragma unroll
            for (int q = 0; q < 32; ++q)
              if (cc + q < p.k) yb = max(yb, a[q] & 0x7fffffffu);
            if (cc + 32 <= p.k && (p.k % 4) == 0) {
#pragma unroll
              for (int q = 0; q < 32; q += 4)
                *reinterpret_cast<float4*>(dst + q) = make_float4(y[q], y[q + 1], y[q + 2], y[q + 3]);
            } else {
#pragma unroll
              for (int q = 0; q < 32; ++q)
                if (cc + q < p.k) dst[q] = y[q];
            }
          }
        }
        ptx::tc_fence_before();
        __syncwarp();
        if (lane == 0) ptx::mbar_arrive(&acce[ab]);
      }
    }
    if (p.ymax) {
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) yb = max(yb, __shfl_xor_sync(0xffffffffu, yb, o));
      if (lane == 0 && yb < 0x7f800000u) atomic_max_nonneg(p.ymax, __uint_as_float(yb));
    }
  }
  __syncthreads();
  if (warp == sk::MMA_W) {
    ptx::tc_fence_after();
    ptx::tmem_dealloc(tmem, 512);
  }
}

template <int NT, int PV>
static void launch_tmem_a(Launcher& L, const Params& p) {
  using C = SkCfg<NT, PV>;
  cudaFuncSetAttribute(tmem_a_kernel<NT, PV>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::SMEM);
  const int64_t tiles = (p.m + 127) / 128;
  const int grid = (int)(tiles < L.num_sms ? (tiles > 0 ? tiles : 1) : L.num_sms);
  tmem_a_kernel<NT, PV><<<grid, sk::THREADS, C::SMEM, L.stream>>>(p);
  L.count(1);
}

// Whether the tensor-memory kernel takes this FP32 X: one matrix, k <= 128,
// 32-byte aligned rows and n a multiple of 8 (whole 32-byte loads).
static bool tmem_a_ok(const Params& p, int nt) {
  return nt <= 2 && !p.units && ((uintptr_t)p.X % 32) == 0 && (p.ldx % 8) == 0 && (p.n % 8) == 0;
}

// V (n x k FP32) -> per k-step tiles [v0 | v1 | v2] of three exact BF16
// pieces (v = v0 + v1 + v2: the top 8 significand bits, then the top 8 of the
// exact remainder, then the rest), in the MN-major SW128 layout of
// tile_v_kernel, zero padded to NPAD columns and to whole k-steps.
__global__ void tile_v3_kernel(const float* __restrict__ V, int64_t n, int k, int npad, uint8_t* __restrict__ out) {
  const int nt = npad / 64;
  const int nks = (int)((n + BK - 1) / BK);
  const uint32_t sbo = nt * 1024;
  const size_t part = (size_t)BK * npad * 2;
  const int64_t total = (int64_t)nks * BK * npad;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int c = (int)(e % npad);
    const int64_t j = e / npad;  // global row of V
    const int ks = (int)(j / BK), kr = (int)(j % BK);
    const float v = (j < n && c < k) ? V[j * k + c] : 0.f;
    const uint32_t b0 = __float_as_uint(v) & 0xffff0000u;
    const float r = v - __uint_as_float(b0);
    const uint32_t b1 = __float_as_uint(r) & 0xffff0000u;
    const float r2 = r - __uint_as_float(b1);
    uint8_t* base = out + (size_t)ks * 3 * part;
    const uint32_t off = ptx::mn_sw128_offset(kr, c, sbo);
    *reinterpret_cast<uint16_t*>(base + off) = (uint16_t)(b0 >> 16);
    *reinterpret_cast<uint16_t*>(base + part + off) = (uint16_t)(b1 >> 16);
    *reinterpret_cast<uint16_t*>(base + 2 * part + off) = (uint16_t)(__float_as_uint(r2) >> 16);
  }
}

template <int XK, int NT, bool EXACT_V>
static void launch_project(Launcher& L, const Params& p, int max_tiles) {
  using C = Cfg<XK, NT, EXACT_V>;
  cudaFuncSetAttribute(project_kernel<XK, NT, EXACT_V>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::SMEM);
  const int64_t tiles = p.units ? max_tiles : (p.m + 127) / 128;
  const int grid = (int)(tiles < L.num_sms ? (tiles > 0 ? tiles : 1) : L.num_sms);
  project_kernel<XK, NT, EXACT_V><<<grid, C::THREADS, C::SMEM, L.stream>>>(p);
  L.count(1);
}

template <int XK, bool EXACT_V = false>
static void launch_project_nt(Launcher& L, const Params& p, int nt, int max_tiles) {
  switch (nt) {
    case 1: launch_project<XK, 1, EXACT_V>(L, p, max_tiles); break;
    case 2: launch_project<XK, 2, EXACT_V>(L, p, max_tiles); break;
    case 3: launch_project<XK, 3, EXACT_V>(L, p, max_tiles); break;
    default: launch_project<XK, 4, EXACT_V>(L, p, max_tiles); break;
  }
}

}  // namespace tcp

void plan_tc_project(char* base, TcProjectWs& w, int xt, int64_t n, int k) {
  const int npad = (k + 63) / 64 * 64;
  const int64_t nks = (n + tcp::BK - 1) / tcp::BK;
  size_t off = 0;
  auto take = [&](size_t b) {
    off = (off + 255) & ~(size_t)255;
    char* r = base ? base + off : nullptr;
    off += b;
    return r;
  };
  w.vhi = take((size_t)nks * 3 * tcp::BK * npad * 2);  // two-part tiles, or three for the FP32 TMEM path
  w.vlo = take(256);  // scalars: [0] max|V|, [1] t
  w.bytes = off + 256;
  (void)xt;
}

namespace tcp {
static void launch_xt(Launcher& L, const Params& p, int xt, int nt, int max_tiles, bool exact_v) {
  // FP32 X against an exact V (the sketch with the very sparse Omega): A in TMEM
  if (exact_v && xt == LSPCA_F32 && tmem_a_ok(p, nt)) {
    if (nt == 1) launch_tmem_a<1, 1>(L, p);
    else launch_tmem_a<2, 1>(L, p);
    return;
  }
  if (exact_v) {
    if (xt == LSPCA_F32) launch_project_nt<XK_F32, true>(L, p, nt, max_tiles);
    else if (xt == LSPCA_BF16) launch_project_nt<XK_BF16, true>(L, p, nt, max_tiles);
    else launch_project_nt<XK_E4M3, true>(L, p, nt, max_tiles);
  } else {
    if (xt == LSPCA_F32) launch_project_nt<XK_F32>(L, p, nt, max_tiles);
    else if (xt == LSPCA_BF16) launch_project_nt<XK_BF16>(L, p, nt, max_tiles);
    else launch_project_nt<XK_E4M3>(L, p, nt, max_tiles);
  }
}
}  // namespace tcp

void tc_project(Launcher& L, const void* X, int xt, int64_t m, int64_t n, int64_t ldx, const float* V, int k,
                TcProjectWs& w, float* Y, int* status, bool exact_v, float* xmax, float* ymax) {
  const int npad = (k + 63) / 64 * 64;
  float* scal = (float*)w.vlo;
  if (tc_xproj_ok(X, xt, ldx, exact_v)) {
    // BF16 / E4M3 X: the TMA-fed kernel; E4M3 takes V as an FP16 pair of V t
    const bool f16 = xt == LSPCA_E4M3;
    cudaMemsetAsync(scal, 0, 8, L.stream);
    if (f16) launch_scan_x(L, V, LSPCA_F32, n, k, k, scal, status);
    const int64_t nks = (n + tcp::BK - 1) / tcp::BK;
    const int64_t total = nks * tcp::BK * npad;
    int blocks = (int)((total + 255) / 256);
    if (blocks > 16 * L.num_sms) blocks = 16 * L.num_sms;
    tcp::tile_v_kernel<<<blocks, 256, 0, L.stream>>>(V, n, k, npad, f16 ? 1 : 0, scal, scal + 1, (uint8_t*)w.vhi);
    L.count(1);
    if (tc_xproj(L, X, xt, m, n, ldx, w.vhi, scal + 1, k, exact_v, Y, status, ymax, xmax != nullptr)) return;
  }
  {
    // FP32 X against a general V, k <= 128: V in three exact BF16 pieces, A in TMEM
    tcp::Params p{};
    p.X = X;
    p.ldx = ldx;
    p.m = m;
    p.n = n;
    p.k = k;
    p.vt = (const uint8_t*)w.vhi;
    p.Y = Y;
    p.status = status;
    p.xmax = xmax;
    p.ymax = ymax;
    if (xt == LSPCA_F32 && !exact_v && tcp::tmem_a_ok(p, npad / 64)) {
      const int64_t nks = (n + tcp::BK - 1) / tcp::BK;
      const int64_t total = nks * tcp::BK * npad;
      int blocks = (int)((total + 255) / 256);
      if (blocks > 16 * L.num_sms) blocks = 16 * L.num_sms;
      tcp::tile_v3_kernel<<<blocks, 256, 0, L.stream>>>(V, n, k, npad, (uint8_t*)w.vhi);
      L.count(1);
      if (npad == 64) tcp::launch_tmem_a<1, 3>(L, p);
      else tcp::launch_tmem_a<2, 3>(L, p);
      return;
    }
  }
  const bool f16 = xt == LSPCA_F32 && !exact_v;  // FP32 X against an exact V takes BF16 tiles
  cudaMemsetAsync(scal, 0, 8, L.stream);
  if (f16) launch_scan_x(L, V, LSPCA_F32, n, k, k, scal, status);
  {
    const int64_t nks = (n + tcp::BK - 1) / tcp::BK;
    const int64_t total = nks * tcp::BK * npad;
    int blocks = (int)((total + 255) / 256);
    if (blocks > 16 * L.num_sms) blocks = 16 * L.num_sms;
    tcp::tile_v_kernel<<<blocks, 256, 0, L.stream>>>(V, n, k, npad, f16 ? 1 : 0, scal, scal + 1, (uint8_t*)w.vhi);
    L.count(1);
  }
  tcp::Params p{};
  p.X = X;
  p.ldx = ldx;
  p.m = m;
  p.n = n;
  p.k = k;
  p.vt = (const uint8_t*)w.vhi;
  p.vscale = scal + 1;
  p.Y = Y;
  p.status = status;
  p.units = nullptr;
  p.nunits = nullptr;
  p.xmax = xmax;
  p.ymax = ymax;
  tcp::launch_xt(L, p, xt, npad / 64, 0, exact_v);
}

bool tc_xproj_tile_v(Launcher& L, int xt, const float* V, int64_t n, int k, TcProjectWs& w, int* status) {
  if (xt != LSPCA_BF16 && xt != LSPCA_E4M3) return false;
  const int npad = (k + 63) / 64 * 64;
  float* scal = (float*)w.vlo;
  const bool f16 = xt == LSPCA_E4M3;
  cudaMemsetAsync(scal, 0, 8, L.stream);
  if (f16) launch_scan_x(L, V, LSPCA_F32, n, k, k, scal, status);
  const int64_t nks = (n + tcp::BK - 1) / tcp::BK;
  const int64_t total = nks * tcp::BK * npad;
  int blocks = (int)((total + 255) / 256);
  if (blocks > 16 * L.num_sms) blocks = 16 * L.num_sms;
  tcp::tile_v_kernel<<<blocks, 256, 0, L.stream>>>(V, n, k, npad, f16 ? 1 : 0, scal, scal + 1, (uint8_t*)w.vhi);
  L.count(1);
  return true;
}

void tc_project_pretiled(Launcher& L, const void* X, int xt, int64_t m, int64_t n, int64_t ldx, const void* tiles,
                         const float* vscale, int k, float* Y, int* status, bool exact_v, float* xmax,
                         float* ymax) {
  tcp::Params p{};
  p.X = X;
  p.ldx = ldx;
  p.m = m;
  p.n = n;
  p.k = k;
  p.vt = (const uint8_t*)tiles;
  p.vscale = vscale;
  p.Y = Y;
  p.status = status;
  p.units = nullptr;
  p.nunits = nullptr;
  p.xmax = xmax;
  p.ymax = ymax;
  tcp::launch_xt(L, p, xt, (k + 63) / 64, 0, exact_v);
}

size_t tc_tile_v_bytes(int64_t n, int k) {
  const int npad = (k + 63) / 64 * 64;
  return (size_t)((n + tcp::BK - 1) / tcp::BK) * 2 * tcp::BK * npad * 2;
}

void tc_tile_v(Launcher& L, int xt, const float* V, int64_t n, int k, void* tiles, float* scal, int* status,
               bool exact_v) {
  const int npad = (k + 63) / 64 * 64;
  const bool f16 = xt == LSPCA_F32 && !exact_v;  // FP32 X against an exact V takes BF16 tiles
  cudaMemsetAsync(scal, 0, 8, L.stream);
  if (f16) launch_scan_x(L, V, LSPCA_F32, n, k, k, scal, status);
  const int64_t nks = (n + tcp::BK - 1) / tcp::BK;
  const int64_t total = nks * tcp::BK * npad;
  int blocks = (int)((total + 255) / 256);
  if (blocks > 16 * L.num_sms) blocks = 16 * L.num_sms;
  tcp::tile_v_kernel<<<blocks, 256, 0, L.stream>>>(V, n, k, npad, f16 ? 1 : 0, scal, scal + 1, (uint8_t*)tiles);
  L.count(1);
}

void tc_project_batch(Launcher& L, int xt, int k, const TcProjUnit* d_units, const int* d_count, int max_tiles,
                      int* status) {
  tcp::Params p{};
  p.units = d_units;
  p.nunits = d_count;
  p.status = status;
  tcp::launch_xt(L, p, xt, (k + 63) / 64, max_tiles, false);
}

}  // namespace lspca
