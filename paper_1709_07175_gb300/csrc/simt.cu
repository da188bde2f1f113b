// Plain SIMT kernels: a tiled GEMM with split-K partials (the FP64 path, the
// cross-check path and the small FP64 products of the k x k step), and the
// fixed-order FP64 reduction of split partials.
#include "common.cuh"
#include "kernels.h"

namespace lspca {

// Load element i of a buffer of run-time type dt, as Acc.
template <typename Acc>
__device__ __forceinline__ Acc ld_any(const void* p, int dt, int64_t i) {
  switch (dt) {
    case LSPCA_F64: return (Acc)((const double*)p)[i];
    case LSPCA_F32: return (Acc)((const float*)p)[i];
    case LSPCA_BF16: return (Acc)__bfloat162float(((const __nv_bfloat16*)p)[i]);
    default: return (Acc)float(((const __nv_fp8_e4m3*)p)[i]);
  }
}

// Tile TS x TS of C per block, BK = 16, 256 threads, (TS/16)^2 outputs each.
// Products of a BK slab are summed first and then added to the running sum
// (two-level summation keeps FP32 rounding at ~sqrt(K/16) + 4 roundings).
template <typename Acc, typename TC, int TS>
__global__ void __launch_bounds__(256) gemm_simt_kernel(int64_t M, int64_t N, int64_t K, const void* __restrict__ A,
                                                        int ta, int64_t lda, int a_trans, const void* __restrict__ B, int tb, int64_t ldb,
                                                        int b_trans, TC* __restrict__ C, int64_t ldc,
                                                        int64_t c_split_stride, int64_t kchunk) {
  constexpr int BK = 16;
  constexpr int TM = TS / 16;
  __shared__ Acc As[BK][TS + 1];
  __shared__ Acc Bs[BK][TS + 1];
  const int tid = threadIdx.x;
  const int tx = tid % 16, ty = tid / 16;
  const int64_t m0 = (int64_t)blockIdx.x * TS;
  const int64_t n0 = (int64_t)blockIdx.y * TS;
  const int64_t kb = (int64_t)blockIdx.z * kchunk;
  const int64_t ke = min(K, kb + kchunk);
  Acc acc[TM][TM];
#pragma unroll
  for (int i = 0; i < TM; ++i)
#pragma unroll
    for (int j = 0; j < TM; ++j) acc[i][j] = Acc(0);
  for (int64_t k0 = kb; k0 < ke; k0 += BK) {
    for (int e = tid; e < BK * TS; e += 256) {
      int r, kk;
      if (a_trans) { r = e % TS; kk = e / TS; } else { kk = e % BK; r = e / BK; }
      const int64_t gr = m0 + r, gk = k0 + kk;
      Acc v = Acc(0);
      if (gr < M && gk < ke) v = ld_any<Acc>(A, ta, a_trans ? gk * lda + gr : gr * lda + gk);
      As[kk][r] = v;
    }
    for (int e = tid; e < BK * TS; e += 256) {
      int c, kk;
      if (b_trans) { kk = e % BK; c = e / BK; } else { c = e % TS; kk = e / TS; }
      const int64_t gc = n0 + c, gk = k0 + kk;
      Acc v = Acc(0);
      if (gc < N && gk < ke) v = ld_any<Acc>(B, tb, b_trans ? gc * ldb + gk : gk * ldb + gc);
      Bs[kk][c] = v;
    }
    __syncthreads();
    Acc part[TM][TM];
#pragma unroll
    for (int i = 0; i < TM; ++i)
#pragma unroll
      for (int j = 0; j < TM; ++j) part[i][j] = Acc(0);
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      Acc a[TM], b[TM];
#pragma unroll
      for (int i = 0; i < TM; ++i) a[i] = As[kk][ty * TM + i];
#pragma unroll
      for (int j = 0; j < TM; ++j) b[j] = Bs[kk][tx * TM + j];
#pragma unroll
      for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int j = 0; j < TM; ++j) part[i][j] = fma(a[i], b[j], part[i][j]);
    }
#pragma unroll
    for (int i = 0; i < TM; ++i)
#pragma unroll
      for (int j = 0; j < TM; ++j) acc[i][j] += part[i][j];
    __syncthreads();
  }
  TC* Cs = C + (int64_t)blockIdx.z * c_split_stride;
#pragma unroll
  for (int i = 0; i < TM; ++i) {
    const int64_t gr = m0 + ty * TM + i;
    if (gr >= M) continue;
#pragma unroll
    for (int j = 0; j < TM; ++j) {
      const int64_t gc = n0 + tx * TM + j;
      if (gc < N) Cs[gr * ldc + gc] = (TC)acc[i][j];
    }
  }
}

template <typename Acc, typename TC>
static void gemm_dispatch_tiles(Launcher& L, int64_t M, int64_t N, int64_t K, const void* A, int ta, int64_t lda,
                                bool at, const void* B, int tb, int64_t ldb, bool bt, void* C, int64_t ldc, int64_t css,
                                int splits, bool small) {
  const int64_t kchunk = ((K + splits - 1) / splits + 15) / 16 * 16;
  if (small) {
    dim3 grid((unsigned)((M + 15) / 16), (unsigned)((N + 15) / 16), (unsigned)splits);
    gemm_simt_kernel<Acc, TC, 16><<<grid, 256, 0, L.stream>>>(M, N, K, A, ta, lda, at, B, tb, ldb, bt, (TC*)C, ldc,
                                                               css, kchunk);
  } else {
    dim3 grid((unsigned)((M + 63) / 64), (unsigned)((N + 63) / 64), (unsigned)splits);
    gemm_simt_kernel<Acc, TC, 64><<<grid, 256, 0, L.stream>>>(M, N, K, A, ta, lda, at, B, tb, ldb, bt, (TC*)C, ldc,
                                                               css, kchunk);
  }
  L.count(1);
}

void launch_gemm_simt(Launcher& L, int64_t M, int64_t N, int64_t K, const void* A, int ta, int64_t lda, bool a_trans,
                      const void* B, int tb, int64_t ldb, bool b_trans, void* C, bool c_f64, int64_t ldc,
                      int64_t c_split_stride, int splits, bool acc_f64, bool small_tiles) {
  if (acc_f64) {
    if (c_f64)
      gemm_dispatch_tiles<double, double>(L, M, N, K, A, ta, lda, a_trans, B, tb, ldb, b_trans, C, ldc, c_split_stride,
                                          splits, small_tiles);
    else
      gemm_dispatch_tiles<double, float>(L, M, N, K, A, ta, lda, a_trans, B, tb, ldb, b_trans, C, ldc, c_split_stride,
                                         splits, small_tiles);
  } else {
    if (c_f64)
      gemm_dispatch_tiles<float, double>(L, M, N, K, A, ta, lda, a_trans, B, tb, ldb, b_trans, C, ldc, c_split_stride,
                                         splits, small_tiles);
    else
      gemm_dispatch_tiles<float, float>(L, M, N, K, A, ta, lda, a_trans, B, tb, ldb, b_trans, C, ldc, c_split_stride,
                                        splits, small_tiles);
  }
}

__global__ void reduce_splits_kernel(const double* __restrict__ part, int splits, int64_t stride, int64_t count,
                                     double* __restrict__ out) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < count; e += (int64_t)gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int q = 0; q < splits; ++q) s += part[q * stride + e];
    out[e] = s;
  }
}

void launch_reduce_splits(Launcher& L, const double* part, int splits, int64_t stride, int64_t count, double* out) {
  const int threads = 256;
  int blocks = (int)((count + threads - 1) / threads);
  if (blocks > 8 * L.num_sms) blocks = 8 * L.num_sms;
  if (blocks < 1) blocks = 1;
  reduce_splits_kernel<<<blocks, threads, 0, L.stream>>>(part, splits, stride, count, out);
  L.count(1);
}

}  // namespace lspca
