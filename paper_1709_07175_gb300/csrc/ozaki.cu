// H = F F^T (the first product of the k x k step, table footnote of Sec. III)
// on the BF16 tensor cores, with the FP64 result an FP64 GEMM would give.
//
// GB300 issues FP64 at about 1/64 of its FP32 rate, so the FP64 product of a
// k x n matrix with its transpose costs milliseconds at k = 256.  Here each
// row of F is cut into fixed-point digits that BF16 holds exactly (Ozaki's
// error-free splitting), the tensor core multiplies digit planes exactly, and
// the digit products are summed in integers:
//
//   1. oz_split_kernel (one CTA per row r): e_r = the row's largest binary
//      exponent, so every a = F[r][q] / 2^e_r lies in (-1, 1); |a| is read as
//      a 63-bit fixed-point integer (from the FP64 bits, no FP64 arithmetic),
//      rounded to 56 bits and cut into eight 7-bit digits, balanced to
//      d_0 in [-128, 128] and d_t in [-64, 64] (t >= 1), with
//      |a - sum_t d_t 2^(-7 (t + 1))| <= 2^-57.  Digit plane t is written as
//      BF16 (exact: integers up to 256) in the 128-byte-swizzled K-major
//      tcgen05 layout, 64 columns of F per block.
//   2. oz_mma_kernel: tile (128 rows x 32 columns of H) x K split.  For every
//      64-column block it multiplies the digit planes of the row tile and
//      the column tile, pairs (t, u) with t + u <= 7, accumulating the pairs
//      of one s = t + u in one TMEM accumulator.  Every product is an integer
//      of at most 2^14 and one column adds at most 10 * 2^12 to an
//      accumulator, so over 256 columns (4 blocks) every partial sum is an
//      integer below 2^24 and the FP32 accumulation is exact.  After 4
//      blocks the epilogue moves the accumulators into 64-bit integers,
//      hi = sum_{s<=3} acc_s 2^(7 (3 - s)), lo = sum_{s>=4} acc_s 2^(7 (7 - s)),
//      while the tensor core fills the other accumulator set.
//   3. oz_fin_kernel: sums the splits' integers (exact, so in any order) and
//      writes H[i][j] = H[j][i] = 2^(e_i + e_j - 63) (hi 2^28 + lo), one
//      rounding (|hi| stays below about n 2^35, so it converts to FP64
//      exactly for n < 2^18; the int64 sums cannot overflow for n < 2^27).
//
// The digits drop below 2^-57 of each row's largest entry and the pairs
// t + u >= 8 (below 2^-55 of the product of the two rows' scales); the rest
// is exact up to the final rounding.  Entries smaller than 2^-57 of their
// row's largest one contribute nothing, as they would contribute below the
// rounding of the largest terms of an FP64 sum.  Subnormal entries count as
// zero; a row holding Inf or NaN makes its row and column of H NaN.
#include "common.cuh"
#include "kernels.h"
#include "tc_ptx.cuh"

namespace lspca {
namespace {

constexpr int kDig = 8;                       // digits per value
constexpr int kBK = 64;                       // columns of F per block
constexpr int kMT = 128, kNT = 32;            // H tile
constexpr int kChunk = 4;                     // blocks per exact accumulation
constexpr uint32_t kAPlane = kMT * kBK * 2;   // 16 KB
constexpr uint32_t kBPlane = kNT * kBK * 2;   // 4 KB
constexpr uint32_t kStage = kDig * (kAPlane + kBPlane);
constexpr int kAccCols = kDig * kNT;          // one accumulator set: 8 x 32 columns
constexpr int kThreads = 192;                 // warps 0-3 epilogue, 4 producer, 5 MMA
constexpr int kNonFinite = 0x7fffffff;
constexpr uint64_t kWaitNs = 2000000000ull;
constexpr uint64_t kDrainNs = 100000000ull;

__host__ __device__ inline int oz_tiles(int kpad) { return kpad == 128 ? 4 : 12; }

// Tiles of the upper triangle: row tile 0 takes every column tile, row tile 1
// (kpad = 256) the column tiles 4..7.
__device__ __forceinline__ void tile_mn(int ti, int kpad, int& mt, int& nt) {
  if (ti < kpad / kNT) {
    mt = 0;
    nt = ti;
  } else {
    mt = 1;
    nt = 4 + (ti - kpad / kNT);
  }
}
__device__ __forceinline__ int tile_of(int mt, int nt) { return mt == 0 ? nt : 8 + (nt - 4); }

// Balanced digits of the FP64 value with bits b in a row whose largest biased
// exponent is E (1 <= E <= 2046): value / 2^(E - 1022) = sum_t d[t] 2^(-7 (t + 1)).
__device__ __forceinline__ void digits(uint64_t b, uint32_t E, int (&d)[kDig]) {
  const uint32_t ee = (uint32_t)(b >> 52) & 0x7ffu;
#pragma unroll
  for (int t = 0; t < kDig; ++t) d[t] = 0;
  if (ee == 0) return;  // zero or subnormal
  const uint64_t mant = (b & 0xfffffffffffffull) | (1ull << 52);
  const int sh = (int)ee - (int)E + 10;  // |value| / 2^(E - 1022) * 2^63 = mant * 2^sh, sh <= 10
  const uint64_t Q = sh >= 0 ? (mant << sh) : (sh > -64 ? (mant >> (-sh)) : 0ull);
  const uint64_t g = (Q + 64u) >> 7;  // 56 bits, rounded to nearest (Q < 2^63 - 2^9: no overflow)
#pragma unroll
  for (int t = 0; t < kDig; ++t) d[t] = (int)((g >> (7 * (kDig - 1 - t))) & 127u);
#pragma unroll
  for (int t = kDig - 1; t >= 1; --t)
    if (d[t] >= 64) {
      d[t] -= 128;
      d[t - 1] += 1;
    }
  if (b >> 63) {
#pragma unroll
    for (int t = 0; t < kDig; ++t) d[t] = -d[t];
  }
}

__global__ void __launch_bounds__(256) oz_split_kernel(const double* __restrict__ F, int k, int64_t n, int nkb,
                                                       int kpad, uint8_t* __restrict__ Dg, int32_t* __restrict__ ex) {
  pdl_wait();  // first, on every path: completion stays ordered along the chain
  __shared__ uint32_t wmax[8];
  const int r = blockIdx.x, tid = threadIdx.x;
  const uint64_t* row = reinterpret_cast<const uint64_t*>(F + (int64_t)r * n);
  uint32_t em = 0;
  if (r < k)
    for (int64_t q = tid; q < n; q += 256) em = max(em, (uint32_t)(row[q] >> 52) & 0x7ffu);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) em = max(em, __shfl_xor_sync(0xffffffffu, em, o));
  if ((tid & 31) == 0) wmax[tid >> 5] = em;
  __syncthreads();
  uint32_t E = 0;
#pragma unroll
  for (int w = 0; w < 8; ++w) E = max(E, wmax[w]);
  if (tid == 0) ex[r] = E == 0x7ffu ? kNonFinite : (E == 0 ? 0 : (int)E - 1022);
  const bool zero_row = r >= k || E == 0 || E == 0x7ffu;
  // one 8-column chunk (one 16-byte line of each plane) per thread and step
  for (int64_t c = tid; c < (int64_t)nkb * 8; c += 256) {
    uint32_t w[kDig][4];
#pragma unroll
    for (int p = 0; p < 4; ++p) {
      int d0[kDig], d1[kDig];
      const int64_t q = c * 8 + 2 * p;
      if (zero_row || q >= n) {
#pragma unroll
        for (int t = 0; t < kDig; ++t) d0[t] = 0;
      } else {
        digits(row[q], E, d0);
      }
      if (zero_row || q + 1 >= n) {
#pragma unroll
        for (int t = 0; t < kDig; ++t) d1[t] = 0;
      } else {
        digits(row[q + 1], E, d1);
      }
#pragma unroll
      for (int t = 0; t < kDig; ++t) {
        const __nv_bfloat162 h = __floats2bfloat162_rn((float)d0[t], (float)d1[t]);
        w[t][p] = *reinterpret_cast<const uint32_t*>(&h);
      }
    }
    const int kb = (int)(c >> 3), j = (int)(c & 7);
#pragma unroll
    for (int t = 0; t < kDig; ++t) {
      uint8_t* dst = Dg + ((size_t)(t * nkb + kb) * kpad + r) * 128 + ((j ^ (r & 7)) << 4);
      *reinterpret_cast<uint4*>(dst) = make_uint4(w[t][0], w[t][1], w[t][2], w[t][3]);
    }
  }
}

// One CTA per (tile, K split); blocks [sp kbpc, min(nkb, (sp + 1) kbpc)).
// Partials: Phi / Plo [split][tile][128 rows][32 columns] int64.
__global__ void __launch_bounds__(kThreads, 1) oz_mma_kernel(const uint8_t* __restrict__ Dg, int nkb, int kpad,
                                                             int kbpc, long long* __restrict__ Phi,
                                                             long long* __restrict__ Plo, int* status) {
  pdl_wait();  // first, on every path: completion stays ordered along the chain
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + kStage);
  uint64_t* empty = full + 1;
  uint64_t* accf = empty + 1;  // [2]
  uint64_t* acce = accf + 2;   // [2]
  uint64_t* drain = acce + 2;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(drain + 1);
  int* abort_flag = reinterpret_cast<int*>(tmem_slot + 1);

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int ti = blockIdx.x, sp = blockIdx.y, tiles = gridDim.x;
  int mt, nt;
  tile_mn(ti, kpad, mt, nt);
  const int kb0 = sp * kbpc;
  const int nk = min(nkb, kb0 + kbpc) - kb0;
  const int nchunks = (nk + kChunk - 1) / kChunk;

  if (tid == 0) {
    ptx::mbar_init(full, 1);
    ptx::mbar_init(empty, 1);
    for (int b = 0; b < 2; ++b) {
      ptx::mbar_init(&accf[b], 1);
      ptx::mbar_init(&acce[b], 4);
    }
    ptx::mbar_init(drain, 1);
    *abort_flag = 0;
    ptx::fence_mbar_init();
  }
  if (warp == 5) ptx::tmem_alloc(tmem_slot, 512);
  ptx::tc_fence_before();
  __syncthreads();
  ptx::tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  const uint32_t sA = ptx::smem_u32(smem), sB = sA + kDig * kAPlane;
  auto fail = [&]() {
    atomicOr(status, ST_TIMEOUT);
    atomicExch(abort_flag, 1);
  };
  auto aborted = [&]() { return *(volatile int*)abort_flag != 0; };

  if (warp == 4) {
    // ------------------------------------------------------------ producer
    if (lane == 0) {
      int i = 0;
      for (; i < nk; ++i) {
        if (!ptx::mbar_wait(empty, (uint32_t)(i & 1) ^ 1u, kWaitNs)) {
          fail();
          break;
        }
        if (aborted()) break;
        ptx::mbar_arrive_expect_tx(full, kStage);
        const int kb = kb0 + i;
#pragma unroll 1
        for (int t = 0; t < kDig; ++t) {
          const uint8_t* plane = Dg + (size_t)(t * nkb + kb) * kpad * 128;
          ptx::bulk_g2s(sA + t * kAPlane, plane + (size_t)mt * kMT * 128, kAPlane, full);
          ptx::bulk_g2s(sB + t * kBPlane, plane + (size_t)nt * kNT * 128, kBPlane, full);
        }
      }
      // bounded wait for the last stage's copies (in flight after an abort)
      if (i > 0) ptx::mbar_wait(full, (uint32_t)((i - 1) & 1), kDrainNs);
    }
    __syncwarp();
  } else if (warp == 5) {
    // ------------------------------------------------------------ MMA issuer
    if (lane == 0) {
      constexpr uint32_t idesc = ptx::idesc_f16(1, kMT, kNT, 0, 0);
      bool ok = true;
      for (int i = 0; i < nk && ok; ++i) {
        const int c = i / kChunk, b = c & 1;
        const bool cstart = (i % kChunk) == 0;
        if (cstart) {
          // the epilogue has drained the chunk that last used accumulator set b
          if (!ptx::mbar_wait(&acce[b], (uint32_t)((c >> 1) & 1) ^ 1u, kWaitNs)) {
            fail();
            ok = false;
            break;
          }
          ptx::tc_fence_after();
        }
        if (!ptx::mbar_wait(full, (uint32_t)(i & 1), kWaitNs) || aborted()) {
          if (!aborted()) fail();
          ok = false;
          break;
        }
        ptx::tc_fence_after();
#pragma unroll 1
        for (int s = 0; s < kDig; ++s) {
          const uint32_t d = tmem + (uint32_t)(b * kAccCols + s * kNT);
#pragma unroll 1
          for (int t = 0; t <= s; ++t) {
            const uint64_t ad = ptx::desc_sw128(sA + t * kAPlane, 16, 1024);
            const uint64_t bd = ptx::desc_sw128(sB + (s - t) * kBPlane, 16, 1024);
#pragma unroll
            for (int kk = 0; kk < kBK / 16; ++kk)
              ptx::mma_f16(d, ptx::desc_advance(ad, kk * 32), ptx::desc_advance(bd, kk * 32), idesc,
                           (cstart && t == 0 && kk == 0) ? 0u : 1u);
          }
        }
        ptx::mma_commit(empty);
        if ((i % kChunk) == kChunk - 1 || i == nk - 1) ptx::mma_commit(&accf[b]);
      }
      ptx::mma_commit(drain);
      if (!ptx::mbar_wait(drain, 0u, kWaitNs)) atomicOr(status, ST_TIMEOUT);
    }
    __syncwarp();
  } else {
    // ------------------------------------------------------------ epilogue
    const uint32_t lane_base = (uint32_t)(32 * warp) << 16;
    const int row = 32 * warp + lane;
    long long hi[kNT], lo[kNT];
#pragma unroll
    for (int q = 0; q < kNT; ++q) hi[q] = lo[q] = 0;
    bool ok = true;
    for (int c = 0; c < nchunks; ++c) {
      const int b = c & 1;
      if (!ptx::mbar_wait(&accf[b], (uint32_t)((c >> 1) & 1), kWaitNs) || aborted()) {
        if (!aborted()) fail();
        ok = false;
        break;
      }
      ptx::tc_fence_after();
#pragma unroll 1
      for (int s = 0; s < 4; ++s) {
        uint32_t v[32];
        ptx::tmem_ld32(tmem + lane_base + (uint32_t)(b * kAccCols + s * kNT), v);
        const long long w = 1ll << (7 * (3 - s));
#pragma unroll
        for (int q = 0; q < kNT; ++q) hi[q] += (long long)__float2int_rn(__uint_as_float(v[q])) * w;  // exact integers
      }
#pragma unroll 1
      for (int s = 4; s < kDig; ++s) {
        uint32_t v[32];
        ptx::tmem_ld32(tmem + lane_base + (uint32_t)(b * kAccCols + s * kNT), v);
        const long long w = 1ll << (7 * (7 - s));
#pragma unroll
        for (int q = 0; q < kNT; ++q) lo[q] += (long long)__float2int_rn(__uint_as_float(v[q])) * w;
      }
      ptx::tc_fence_before();
      __syncwarp();
      if (lane == 0) ptx::mbar_arrive(&acce[b]);
    }
    if (ok) {
      const size_t base = (((size_t)sp * tiles + ti) * kMT + row) * kNT;
#pragma unroll
      for (int q = 0; q < kNT; q += 2) {
        *reinterpret_cast<longlong2*>(Phi + base + q) = make_longlong2(hi[q], hi[q + 1]);
        *reinterpret_cast<longlong2*>(Plo + base + q) = make_longlong2(lo[q], lo[q + 1]);
      }
    }
  }
  __syncthreads();
  if (warp == 5) {
    ptx::tc_fence_after();
    ptx::tmem_dealloc(tmem, 512);
  }
}

// H[i][j] = H[j][i] for j >= i from the splits' integer partials.
__global__ void __launch_bounds__(256) oz_fin_kernel(const long long* __restrict__ Phi,
                                                     const long long* __restrict__ Plo,
                                                     const int32_t* __restrict__ ex, int k, int kpad, int splits,
                                                     double* __restrict__ H) {
  pdl_wait();  // first, on every path: completion stays ordered along the chain
  const int tiles = oz_tiles(kpad);
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (int64_t)k * k) return;
  const int i = (int)(e / k), j = (int)(e % k);
  if (j < i) return;
  const int t = tile_of(i / kMT, j / kNT);
  const size_t off = ((size_t)t * kMT + (i % kMT)) * kNT + (j % kNT);
  const size_t stride = (size_t)tiles * kMT * kNT;
  long long sh = 0, sl = 0;
  for (int s = 0; s < splits; ++s) {
    sh += Phi[s * stride + off];
    sl += Plo[s * stride + off];
  }
  const int ei = ex[i], ej = ex[j];
  double v;
  if (ei == kNonFinite || ej == kNonFinite) v = __longlong_as_double(0x7ff8000000000000ll);
  else v = ldexp(fma((double)sh, 0x1p28, (double)sl), ei + ej - 63);
  H[(int64_t)i * k + j] = v;
  H[(int64_t)j * k + i] = v;
}

struct OzPlan {
  int kpad, nkb, tiles, kbpc, splits;
};

OzPlan oz_plan(int k, int64_t n) {
  OzPlan p;
  p.kpad = k <= 128 ? 128 : 256;
  p.nkb = (int)((n + kBK - 1) / kBK);
  if (p.nkb < 1) p.nkb = 1;
  p.tiles = oz_tiles(p.kpad);
  const int64_t units = (int64_t)p.tiles * p.nkb;
  p.kbpc = (int)((units + 159) / 160);
  if (p.kbpc < 1) p.kbpc = 1;
  p.splits = (p.nkb + p.kbpc - 1) / p.kbpc;
  return p;
}

size_t align_up(size_t b) { return (b + 255) & ~(size_t)255; }

}  // namespace

size_t oz_gram_ws_bytes(int k, int64_t n) {
  const OzPlan p = oz_plan(k, n);
  return align_up((size_t)kDig * p.nkb * p.kpad * 128) + align_up((size_t)p.kpad * 4) +
         2 * align_up((size_t)p.splits * p.tiles * kMT * kNT * 8) + 256;
}

void launch_oz_gram(Launcher& L, const double* F, int k, int64_t n, void* ws, double* H, int* status) {
  const OzPlan p = oz_plan(k, n);
  uint8_t* base = (uint8_t*)(((uintptr_t)ws + 255) & ~(uintptr_t)255);
  uint8_t* Dg = base;
  base += align_up((size_t)kDig * p.nkb * p.kpad * 128);
  int32_t* ex = (int32_t*)base;
  base += align_up((size_t)p.kpad * 4);
  long long* Phi = (long long*)base;
  base += align_up((size_t)p.splits * p.tiles * kMT * kNT * 8);
  long long* Plo = (long long*)base;
  launch_pdl(L, oz_split_kernel, dim3(p.kpad), dim3(256), 0, F, k, n, p.nkb, p.kpad, Dg, ex);
  const size_t smem = kStage + 1024 + 128;
  cudaFuncSetAttribute(oz_mma_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  launch_pdl(L, oz_mma_kernel, dim3(p.tiles, p.splits), dim3(kThreads), smem, (const uint8_t*)Dg, p.nkb, p.kpad,
             p.kbpc, Phi, Plo, status);
  const int64_t kk = (int64_t)k * k;
  launch_pdl(L, oz_fin_kernel, dim3((unsigned)((kk + 255) / 256)), dim3(256), 0, (const long long*)Phi,
             (const long long*)Plo, (const int32_t*)ex, k, p.kpad, p.splits, H);
  L.count(3);
}

}  // namespace lspca
