// Tensor-core pass F (Algorithm 4's F += U_s^T X_s) on sm_103a with tcgen05/TMEM.
//
// D[c, j] = sum over the rows i of one m-chunk of U[i, c] X[i, j]: a GEMM whose
// reduction runs over the rows of two row-major sources (U is m x k, X is m x n),
// so both operands are MN-major.  M = k (one or two 128-row halves), N = a
// 256-column (128 when k > 128) tile of X, K = rows.
//
// Number formats.  FP32 X: both operands are split into FP16 pairs
// v s = hi + lo (hi = fp16(v s), lo = fp16(v s - hi)) with power-of-two scales
// s chosen from max|X| and max|U| so that |v s| <= 2^14; the three products
// hi*hi + hi*lo + lo*hi carry ~22 significant bits (FP16 pairs keep 3 more
// bits per piece than BF16 pairs).  BF16 X: X is exact, U is split into a BF16
// pair, two products.
//
// Accumulation.  Measured on GB300, the FP32 accumulation of tcgen05.mma into
// TMEM behaves like round-toward-zero: its error is biased and grows linearly
// with the number of accumulating instructions (a Gram U^T U over 512 rows came
// out uniformly smaller by 2.6e-6).  So the tensor core only accumulates short
// segments of SEG k-steps (SEG * BK rows) into TMEM region A; the epilogue warps
// add each finished segment into a round-to-nearest FP32 running sum S kept in
// TMEM region B (S = A for a unit's first segment), and write S as the unit's
// FP32 partial after its last segment.  Partials of the m-chunks are summed in
// FP64 in fixed order.
//
// Kernel structure (one persistent CTA per SM, 13 warps):
//   warps 0-7   converters: 16-byte global loads of the U and X rows of a
//               K-step (kept one step ahead in registers), split/convert, and
//               store into the 128-byte-swizzled MN-major layout;
//   warps 8-11  epilogue: fold each finished segment into the running sum
//               (tcgen05.ld / tcgen05.st), scale and write the unit's partial;
//   warp 12     TMEM allocation and the single thread that issues tcgen05.mma
//               and tcgen05.commit.
// A 4-stage shared-memory ring (mbarriers full/empty) feeds the MMAs; the
// segment accumulator A is handed between the MMA thread and the epilogue with
// the mbarriers accf / acce.
// Every mbarrier wait is bounded (2 s of %globaltimer): on expiry the kernel
// records ST_TIMEOUT, stops issuing work, waits for its MMAs and frees TMEM.
#include <type_traits>

#include "common.cuh"
#include "tc.h"
#include "tc_ptx.cuh"

namespace lspca {

bool tc_available() {
  int dev = 0, maj = 0, min = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return false;
  cudaDeviceGetAttribute(&maj, cudaDevAttrComputeCapabilityMajor, dev);
  cudaDeviceGetAttribute(&min, cudaDevAttrComputeCapabilityMinor, dev);
  return maj == 10 && min == 3;
}

namespace tcc {

constexpr int BK = 32;              // rows (K) per pipeline stage
constexpr int STAGES = 4;
constexpr int CONV_WARPS = 8;
constexpr int CONV_THREADS = CONV_WARPS * 32;
constexpr int EPI_WARP0 = 8;
constexpr int MMA_WARP = 12;
constexpr int THREADS = 13 * 32;
constexpr uint64_t kWaitNs = 2000000000ull;
constexpr int SEG = 4;               // k-steps accumulated by the tensor core per segment

enum XKind { XK_F32 = 0, XK_BF16 = 1, XK_E4M3 = 2 };

struct Params {
  const float* U;      // m x k, ld ldu (A source)
  int64_t ldu;
  const void* B;       // m x nb source of the B operand (X, or U for the Gram)
  int64_t ldb;
  int64_t nb;          // columns of the B source
  int64_t m;
  int k;
  int tiles;           // N tiles of the B source
  int chunks;          // m-chunks
  int64_t rows_per_chunk;
  float* part;         // chunks x k x nb FP32 partials
  const float* amax_b; // max|B source| (device), FP32 path
  const float* amax_u; // max|U| (device), FP32 path
  int* status;
};

template <int XK, int MH>
struct Cfg {
  static constexpr int BN = 256 / MH;
  static constexpr int WA = 128 * MH;
  static constexpr int NB = (XK == XK_F32) ? 2 : 1;        // B operand parts
  static constexpr uint32_t A_BYTES = BK * WA * 2;
  static constexpr uint32_t B_BYTES = BK * BN * 2;
  static constexpr uint32_t SBO_A = (WA / 64) * 1024;
  static constexpr uint32_t SBO_B = (BN / 64) * 1024;
  static constexpr uint32_t STAGE_BYTES = 2 * A_BYTES + NB * B_BYTES;
  static constexpr int A_VEC = BK * WA / 4 / CONV_THREADS;        // float4 per thread
  static constexpr int B_VEC = (XK == XK_F32)    ? BK * BN / 4 / CONV_THREADS
                               : (XK == XK_BF16) ? BK * BN / 8 / CONV_THREADS
                                                 : BK * BN / 16 / CONV_THREADS;
  // 8 KB of slack after the ring keeps every descriptor-addressed byte inside
  // the allocation
  static constexpr size_t SMEM = 1024 + STAGES * STAGE_BYTES + 256 + 8192;
  static constexpr uint32_t TMEM_COLS = 512;  // segment accumulator A (MH x BN = 256) + running sum S (256)
};

__device__ __forceinline__ float pow2_scale(float amax) {
  if (!(amax > 0.f) || !isfinite(amax)) return 1.f;
  int e;
  frexpf(amax, &e);  // amax < 2^e
  return ldexpf(1.f, 14 - e);
}

template <typename H>
__device__ __forceinline__ void split2(float v, H& hi, H& lo);
template <>
__device__ __forceinline__ void split2<__half>(float v, __half& hi, __half& lo) {
  hi = __float2half_rn(v);
  lo = __float2half_rn(v - __half2float(hi));
}
template <>
__device__ __forceinline__ void split2<__nv_bfloat16>(float v, __nv_bfloat16& hi, __nv_bfloat16& lo) {
  hi = __float2bfloat16_rn(v);
  lo = __float2bfloat16_rn(v - __bfloat162float(hi));
}

template <typename H>
__device__ __forceinline__ uint2 pack4(H a, H b, H c, H d) {
  uint2 r;
  r.x = (uint32_t)(*reinterpret_cast<uint16_t*>(&a)) | ((uint32_t)(*reinterpret_cast<uint16_t*>(&b)) << 16);
  r.y = (uint32_t)(*reinterpret_cast<uint16_t*>(&c)) | ((uint32_t)(*reinterpret_cast<uint16_t*>(&d)) << 16);
  return r;
}

__device__ __forceinline__ void sts64(uint32_t addr, uint2 v) {
  asm volatile("st.shared.v2.b32 [%0], {%1, %2};" ::"r"(addr), "r"(v.x), "r"(v.y) : "memory");
}
__device__ __forceinline__ void sts128(uint32_t addr, uint4 v) {
  asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(addr), "r"(v.x), "r"(v.y), "r"(v.z), "r"(v.w)
               : "memory");
}

__device__ __forceinline__ float4 ldg_stream4(const float* p) {
  float4 v;
  asm volatile("ld.global.nc.L1::no_allocate.v4.f32 {%0, %1, %2, %3}, [%4];"
               : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
               : "l"(p));
  return v;
}
__device__ __forceinline__ uint4 ldg_stream16(const void* p) {
  uint4 v;
  asm volatile("ld.global.nc.L1::no_allocate.v4.u32 {%0, %1, %2, %3}, [%4];"
               : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
               : "l"(p));
  return v;
}

template <int XK, int MH>
__global__ void __launch_bounds__(THREADS, 1) chain_kernel(Params p) {
  using C = Cfg<XK, MH>;
  using H = typename std::conditional<XK == XK_F32, __half, __nv_bfloat16>::type;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + STAGES * C::STAGE_BYTES);
  uint64_t* empty = full + STAGES;
  uint64_t* accf = empty + STAGES;
  uint64_t* acce = accf + 2;
  uint64_t* drain = acce + 2;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(drain + 1);
  int* abort_flag = reinterpret_cast<int*>(tmem_slot + 1);

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int units = p.tiles * p.chunks;

  if (tid == 0) {
    for (int s = 0; s < STAGES; ++s) {
      ptx::mbar_init(&full[s], CONV_WARPS);
      ptx::mbar_init(&empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      ptx::mbar_init(&accf[b], 1);
      ptx::mbar_init(&acce[b], 4);
    }
    ptx::mbar_init(drain, 1);
    *abort_flag = 0;
    ptx::fence_mbar_init();
  }
  if (warp == MMA_WARP) ptx::tmem_alloc(tmem_slot, C::TMEM_COLS);
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

  if (warp < CONV_WARPS) {
    // ------------------------------------------------------------ converters
    float sa = 1.f, sb = 1.f;
    if (XK == XK_F32) {
      sa = pow2_scale(*p.amax_u);
      sb = pow2_scale(*p.amax_b);
    }
    auto load = [&](int64_t i0, int64_t i1, int tile, float4 (&ra)[C::A_VEC], uint4 (&rb)[C::B_VEC]) {
#pragma unroll
      for (int q = 0; q < C::A_VEC; ++q) {
        const int f = tid + CONV_THREADS * q;
        const int kr = f / (C::WA / 4), mn = (f % (C::WA / 4)) * 4;
        const int64_t gi = i0 + kr;
        if (gi < i1 && mn < p.k)
          ra[q] = ldg_stream4(p.U + gi * p.ldu + mn);
        else
          ra[q] = make_float4(0.f, 0.f, 0.f, 0.f);
      }
      const int64_t col0 = (int64_t)tile * C::BN;
#pragma unroll
      for (int q = 0; q < C::B_VEC; ++q) {
        const int f = tid + CONV_THREADS * q;
        if (XK == XK_F32) {
          const int kr = f / (C::BN / 4), mn = (f % (C::BN / 4)) * 4;
          const int64_t gi = i0 + kr, gj = col0 + mn;
          if (gi < i1 && gj < p.nb)
            rb[q] = ldg_stream16((const float*)p.B + gi * p.ldb + gj);
          else
            rb[q] = make_uint4(0u, 0u, 0u, 0u);
        } else if (XK == XK_BF16) {
          const int kr = f / (C::BN / 8), mn = (f % (C::BN / 8)) * 8;
          const int64_t gi = i0 + kr, gj = col0 + mn;
          if (gi < i1 && gj < p.nb)
            rb[q] = ldg_stream16((const __nv_bfloat16*)p.B + gi * p.ldb + gj);
          else
            rb[q] = make_uint4(0u, 0u, 0u, 0u);
        } else {
          const int kr = f / (C::BN / 16), mn = (f % (C::BN / 16)) * 16;
          const int64_t gi = i0 + kr, gj = col0 + mn;
          if (gi < i1 && gj < p.nb)
            rb[q] = ldg_stream16((const uint8_t*)p.B + gi * p.ldb + gj);
          else
            rb[q] = make_uint4(0u, 0u, 0u, 0u);
        }
      }
    };
    auto store = [&](uint32_t stage_addr, const float4 (&ra)[C::A_VEC], const uint4 (&rb)[C::B_VEC]) {
      const uint32_t a_hi = stage_addr, a_lo = stage_addr + C::A_BYTES;
      const uint32_t b_hi = stage_addr + 2 * C::A_BYTES, b_lo = b_hi + C::B_BYTES;
#pragma unroll
      for (int q = 0; q < C::A_VEC; ++q) {
        const int f = tid + CONV_THREADS * q;
        const int kr = f / (C::WA / 4), mn = (f % (C::WA / 4)) * 4;
        H h0, h1, h2, h3, l0, l1, l2, l3;
        split2<H>(ra[q].x * sa, h0, l0);
        split2<H>(ra[q].y * sa, h1, l1);
        split2<H>(ra[q].z * sa, h2, l2);
        split2<H>(ra[q].w * sa, h3, l3);
        const uint32_t off = ptx::mn_sw128_offset(kr, mn, C::SBO_A);
        sts64(a_hi + off, pack4<H>(h0, h1, h2, h3));
        sts64(a_lo + off, pack4<H>(l0, l1, l2, l3));
      }
#pragma unroll
      for (int q = 0; q < C::B_VEC; ++q) {
        const int f = tid + CONV_THREADS * q;
        if (XK == XK_F32) {
          const int kr = f / (C::BN / 4), mn = (f % (C::BN / 4)) * 4;
          const float4 v = *reinterpret_cast<const float4*>(&rb[q]);
          H h0, h1, h2, h3, l0, l1, l2, l3;
          split2<H>(v.x * sb, h0, l0);
          split2<H>(v.y * sb, h1, l1);
          split2<H>(v.z * sb, h2, l2);
          split2<H>(v.w * sb, h3, l3);
          const uint32_t off = ptx::mn_sw128_offset(kr, mn, C::SBO_B);
          sts64(b_hi + off, pack4<H>(h0, h1, h2, h3));
          sts64(b_lo + off, pack4<H>(l0, l1, l2, l3));
        } else if (XK == XK_BF16) {
          const int kr = f / (C::BN / 8), mn = (f % (C::BN / 8)) * 8;
          sts128(b_hi + ptx::mn_sw128_offset(kr, mn, C::SBO_B), rb[q]);
        } else {
          // FP8 E4M3 values widen exactly to BF16
          const int kr = f / (C::BN / 16), mn = (f % (C::BN / 16)) * 16;
          const __nv_fp8_e4m3* e8 = reinterpret_cast<const __nv_fp8_e4m3*>(&rb[q]);
          uint32_t w[8];
#pragma unroll
          for (int u = 0; u < 8; ++u) {
            __nv_bfloat162 h2 = __floats2bfloat162_rn(float(e8[2 * u]), float(e8[2 * u + 1]));
            w[u] = *reinterpret_cast<uint32_t*>(&h2);
          }
          sts128(b_hi + ptx::mn_sw128_offset(kr, mn, C::SBO_B), make_uint4(w[0], w[1], w[2], w[3]));
          sts128(b_hi + ptx::mn_sw128_offset(kr, mn + 8, C::SBO_B), make_uint4(w[4], w[5], w[6], w[7]));
        }
      }
    };
    auto unit_rows = [&](int64_t u, int64_t& i0, int64_t& i1) {
      i0 = (u / p.tiles) * p.rows_per_chunk;
      i1 = i0 + p.rows_per_chunk;
      if (i1 > p.m) i1 = p.m;
    };
    // (unit, k-step) flattened into one stream; the next step's loads are in
    // flight while the current step is converted and stored.
    float4 ra[C::A_VEC], ra_n[C::A_VEC];
    uint4 rb[C::B_VEC], rb_n[C::B_VEC];
    int64_t unit = blockIdx.x, kst = 0, step = 0;
    int64_t c0, c1;
    unit_rows(unit, c0, c1);
    load(c0, c1, (int)(unit % p.tiles), ra, rb);
    while (true) {
      const int64_t nsteps = (c1 - c0 + BK - 1) / BK;
      int64_t nunit = unit, nk = kst + 1;
      if (nk >= nsteps) {
        nunit = unit + gridDim.x;
        nk = 0;
      }
      int64_t n0 = 0, n1 = 0;
      const bool more = nunit < units;
      if (more) {
        unit_rows(nunit, n0, n1);
        load(n0 + nk * BK, n1, (int)(nunit % p.tiles), ra_n, rb_n);
      }
      const int s = (int)(step % STAGES);
      const uint32_t ph = (uint32_t)((step / STAGES) & 1);
      if (!ptx::mbar_wait(&empty[s], ph ^ 1u, kWaitNs)) {
        fail();
        break;
      }
      if (aborted()) break;
      store(sbase + s * C::STAGE_BYTES, ra, rb);
      ptx::fence_proxy_async_smem();
      __syncwarp();
      if (lane == 0) ptx::mbar_arrive(&full[s]);
      ++step;
      if (!more) break;
      unit = nunit;
      kst = nk;
      c0 = n0;
      c1 = n1;
#pragma unroll
      for (int q = 0; q < C::A_VEC; ++q) ra[q] = ra_n[q];
#pragma unroll
      for (int q = 0; q < C::B_VEC; ++q) rb[q] = rb_n[q];
    }
  } else if (warp == MMA_WARP) {
    // ------------------------------------------------------------ MMA issuer
    if (lane == 0) {
      constexpr uint32_t idesc = ptx::idesc_f16(XK == XK_F32 ? 0 : 1, 128, C::BN, 1, 1);
      int64_t step = 0, seg = 0;
      bool ok = true;
      for (int64_t unit = blockIdx.x; unit < units && ok; unit += gridDim.x) {
        const int64_t ch = unit / p.tiles;
        int64_t i0 = ch * p.rows_per_chunk, i1 = i0 + p.rows_per_chunk;
        if (i1 > p.m) i1 = p.m;
        const int64_t nsteps = (i1 - i0 + BK - 1) / BK;
        for (int64_t t = 0; t < nsteps && ok; ++t, ++step) {
          const bool seg_start = (t % SEG) == 0;
          if (seg_start) {
            // wait until the epilogue has folded the previous segment out of A
            if (!ptx::mbar_wait(&acce[0], (uint32_t)((seg & 1) ^ 1), kWaitNs)) {
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
          const uint32_t a_hi = st, a_lo = st + C::A_BYTES, b_hi = st + 2 * C::A_BYTES, b_lo = b_hi + C::B_BYTES;
#pragma unroll
          for (int kk = 0; kk < BK / 16; ++kk) {
            const uint64_t bdh = ptx::desc_sw128(b_hi + kk * 2 * C::SBO_B, 1024, C::SBO_B);
            const uint64_t bdl = ptx::desc_sw128(b_lo + kk * 2 * C::SBO_B, 1024, C::SBO_B);
#pragma unroll
            for (int h = 0; h < MH; ++h) {
              const uint32_t d = tmem + (uint32_t)(h * C::BN);
              const uint64_t adh = ptx::desc_sw128(a_hi + kk * 2 * C::SBO_A + h * 2048, 1024, C::SBO_A);
              const uint64_t adl = ptx::desc_sw128(a_lo + kk * 2 * C::SBO_A + h * 2048, 1024, C::SBO_A);
              const uint32_t acc = (seg_start && kk == 0) ? 0u : 1u;
              ptx::mma_f16(d, adh, bdh, idesc, acc);
              if (XK == XK_F32) ptx::mma_f16(d, adh, bdl, idesc, 1u);
              ptx::mma_f16(d, adl, bdh, idesc, 1u);
            }
          }
          ptx::mma_commit(&empty[s]);
          if ((t % SEG) == SEG - 1 || t == nsteps - 1) {
            ptx::mma_commit(&accf[0]);
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
    const int e = warp - EPI_WARP0;  // TMEM lane quarter
    float sc = 1.f;
    if (XK == XK_F32) sc = 1.f / (pow2_scale(*p.amax_u) * pow2_scale(*p.amax_b));
    const uint32_t lane_base = (uint32_t)(32 * e) << 16;
    constexpr uint32_t S_COL = MH * C::BN;  // running sum S follows the segment accumulator A
    int64_t seg = 0;
    bool ok = true;
    for (int64_t unit = blockIdx.x; unit < units && ok; unit += gridDim.x) {
      const int tile = (int)(unit % p.tiles);
      const int64_t ch = unit / p.tiles;
      int64_t i0 = ch * p.rows_per_chunk, i1 = i0 + p.rows_per_chunk;
      if (i1 > p.m) i1 = p.m;
      const int64_t nsteps = (i1 - i0 + BK - 1) / BK;
      const int64_t nseg = (nsteps + SEG - 1) / SEG;
      for (int64_t g = 0; g < nseg; ++g, ++seg) {
        if (!ptx::mbar_wait(&accf[0], (uint32_t)(seg & 1), kWaitNs) || aborted()) {
          if (!aborted()) fail();
          ok = false;
          break;
        }
        ptx::tc_fence_after();
        const bool first = g == 0, last = g == nseg - 1;
#pragma unroll
        for (int h = 0; h < MH; ++h) {
          const int c = 128 * h + 32 * e + lane;
#pragma unroll 1
          for (int c0 = 0; c0 < C::BN; c0 += 32) {
            const uint32_t col = (uint32_t)(h * C::BN + c0);
            uint32_t a[32], r[32];
            ptx::tmem_ld32(tmem + lane_base + col, a);
            if (first) {
#pragma unroll
              for (int q = 0; q < 32; ++q) r[q] = a[q];
            } else {
              ptx::tmem_ld32(tmem + lane_base + S_COL + col, r);
#pragma unroll
              for (int q = 0; q < 32; ++q) r[q] = __float_as_uint(__uint_as_float(r[q]) + __uint_as_float(a[q]));
            }
            if (!last) {
              ptx::tmem_st32(tmem + lane_base + S_COL + col, r);
            } else if (c < p.k) {
              const int64_t j0 = (int64_t)tile * C::BN + c0;
              float* dst = p.part + (ch * p.k + c) * p.nb + j0;
              if (j0 + 32 <= p.nb) {
#pragma unroll
                for (int q = 0; q < 32; q += 4)
                  *reinterpret_cast<float4*>(dst + q) =
                      make_float4(__uint_as_float(r[q]) * sc, __uint_as_float(r[q + 1]) * sc,
                                  __uint_as_float(r[q + 2]) * sc, __uint_as_float(r[q + 3]) * sc);
              } else {
#pragma unroll
                for (int q = 0; q < 32; ++q)
                  if (j0 + q < p.nb) dst[q] = __uint_as_float(r[q]) * sc;
              }
            }
          }
        }
        ptx::tc_fence_before();
        __syncwarp();
        if (lane == 0) ptx::mbar_arrive(&acce[0]);
      }
    }
  }

  __syncthreads();
  if (warp == MMA_WARP) {
    ptx::tc_fence_after();
    ptx::tmem_dealloc(tmem, C::TMEM_COLS);
  }
}

// FP64 fixed-order sum of FP32 chunk partials.
// Fixed-order sum of FP32 chunk partials into FP64 (out = sum, or out += sum
// with accumulate).  The sum runs in FP32 with Knuth's error-free TwoSum
// carrying the rounding error of every addition (GB300 issues few FP64 adds);
// sum + error is the partials' sum to ~2^-48 relative to their magnitudes.
__global__ void reduce_f32_parts_kernel(const float* __restrict__ part, int chunks, int64_t count,
                                        double* __restrict__ out, int accumulate, const int* gate) {
  if (gate && *gate == 0) return;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < count; e += (int64_t)gridDim.x * blockDim.x) {
    float s = 0.f, c = 0.f;
    // unrolled so the independent loads run ahead of the dependent adds
#pragma unroll 8
    for (int q = 0; q < chunks; ++q) {
      const float x = part[(int64_t)q * count + e];
      const float t = s + x;
      const float bp = t - s;
      c += (s - (t - bp)) + (x - bp);
      s = t;
    }
    const double v = (double)s + (double)c;
    out[e] = accumulate ? out[e] + v : v;
  }
}

template <int XK, int MH>
static void launch_chain(Launcher& L, const Params& p) {
  using C = Cfg<XK, MH>;
  cudaFuncSetAttribute(chain_kernel<XK, MH>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::SMEM);
  const int units = p.tiles * p.chunks;
  const int grid = units < L.num_sms ? units : L.num_sms;
  chain_kernel<XK, MH><<<grid, THREADS, C::SMEM, L.stream>>>(p);
  L.count(1);
}

static void choose_chunks(int64_t m, int tiles, int num_sms, int& chunks, int64_t& rows) {
  // about four units per CTA, chunks of >= 512 rows
  int64_t c = (4LL * num_sms + tiles - 1) / tiles;
  const int64_t cmax = (m + 511) / 512;
  if (c > cmax) c = cmax;
  if (c < 1) c = 1;
  rows = (m + c - 1) / c;
  rows = (rows + BK - 1) / BK * BK;
  chunks = (int)((m + rows - 1) / rows);
}

}  // namespace tcc

void plan_tc_chain_inline(char* base, TcChainWs& w, int xt, int64_t m, int64_t n, int k, bool want_g, int num_sms) {
  const int MH = k > 128 ? 2 : 1;
  const int BN = 256 / MH;
  const int tiles = (int)((n + BN - 1) / BN);
  int chunks;
  int64_t rows;
  tcc::choose_chunks(m, tiles, num_sms, chunks, rows);
  w.chunks = chunks;
  w.rows_per_chunk = rows;
  size_t off = 0;
  auto take = [&](size_t b) {
    off = (off + 255) & ~(size_t)255;
    char* r = base ? base + off : nullptr;
    off += b;
    return r;
  };
  w.Fpart = (double*)take((size_t)chunks * k * n * 4);  // FP32 partials (typed as bytes)
  w.Gpart = nullptr;
  w.gchunks = 0;
  if (want_g) {
    const int gt = (k + BN - 1) / BN;
    int gc;
    int64_t grows;
    tcc::choose_chunks(m, gt, num_sms, gc, grows);
    w.gchunks = gc;
    w.grows_per_chunk = grows;
    w.Gpart = (double*)take((size_t)gc * k * k * 4);
  }
  w.bytes = off + 256;
  (void)xt;
}

void tc_chain_inline_main(Launcher& L, const void* X, int xt, int64_t m, int64_t n, int64_t ldx, const float* U,
                          int k, TcChainWs& w, const float* absmax, int* status, bool want_g) {
  const int MH = k > 128 ? 2 : 1;
  tcc::Params p{};
  p.U = U;
  p.ldu = k;
  p.B = X;
  p.ldb = ldx;
  p.nb = n;
  p.m = m;
  p.k = k;
  p.tiles = (int)((n + 256 / MH - 1) / (256 / MH));
  p.chunks = w.chunks;
  p.rows_per_chunk = w.rows_per_chunk;
  p.part = (float*)w.Fpart;
  p.amax_b = absmax;
  p.amax_u = absmax + 1;
  p.status = status;
  if (xt == LSPCA_F32) {
    if (MH == 1) tcc::launch_chain<tcc::XK_F32, 1>(L, p);
    else tcc::launch_chain<tcc::XK_F32, 2>(L, p);
  } else if (xt == LSPCA_BF16) {
    if (MH == 1) tcc::launch_chain<tcc::XK_BF16, 1>(L, p);
    else tcc::launch_chain<tcc::XK_BF16, 2>(L, p);
  } else {
    if (MH == 1) tcc::launch_chain<tcc::XK_E4M3, 1>(L, p);
    else tcc::launch_chain<tcc::XK_E4M3, 2>(L, p);
  }
  if (want_g) {
    // G = U^T U: the same kernel with U as the B source (FP32 split path)
    tcc::Params g = p;
    g.B = U;
    g.ldb = k;
    g.nb = k;
    g.tiles = (int)((k + 256 / MH - 1) / (256 / MH));
    g.chunks = w.gchunks;
    g.rows_per_chunk = w.grows_per_chunk;
    g.part = (float*)w.Gpart;
    g.amax_b = absmax + 1;
    if (MH == 1) tcc::launch_chain<tcc::XK_F32, 1>(L, g);
    else tcc::launch_chain<tcc::XK_F32, 2>(L, g);
  }
}

void tc_chain_reduce(Launcher& L, int64_t n, int k, TcChainWs& w, double* F, double* G, bool accumulate,
                     const int* gate) {
  const int threads = 256;
  int64_t cnt = (int64_t)k * n;
  int blocks = (int)((cnt + threads - 1) / threads);
  if (blocks > 8 * L.num_sms) blocks = 8 * L.num_sms;
  tcc::reduce_f32_parts_kernel<<<blocks, threads, 0, L.stream>>>((const float*)w.Fpart, w.chunks, cnt, F,
                                                                 accumulate ? 1 : 0, gate);
  L.count(1);
  if (G && w.Gpart) {
    cnt = (int64_t)k * k;
    blocks = (int)((cnt + threads - 1) / threads);
    tcc::reduce_f32_parts_kernel<<<blocks, threads, 0, L.stream>>>((const float*)w.Gpart, w.gchunks, cnt, G,
                                                                   accumulate ? 1 : 0, nullptr);
    L.count(1);
  }
}


}  // namespace lspca
