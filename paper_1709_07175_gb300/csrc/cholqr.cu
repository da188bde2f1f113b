// R factor of the tall-skinny U for the SPCA comparison path (Algorithms 1
// and 3 orthonormalise U by QR and keep only R) by CholeskyQR2:
//   G1 = U^T U (the Gram pass F already forms),  R1 = chol(G1),
//   Q1 = U R1^-1 (the tensor-core reduction map),  G2 = Q1^T Q1,
//   R2 = chol(G2),  R = R2 R1.
// One Cholesky alone loses orthogonality in proportion to cond(U)^2; the
// second pass factors the nearly orthonormal Q1 and restores it to working
// precision whenever the first Cholesky succeeds (cond(U) below about the
// inverse square root of the Gram's precision).  A Cholesky whose pivot
// falls below kPivotTol of its diagonal entry sets a flag, and the
// Householder TSQR (tsqr.cu) then computes R instead; every kernel here
// reads that flag and does nothing once it is set.
#include "common.cuh"
#include "kernels.h"

namespace lspca {
namespace {

constexpr int kCholThreads = 1024;
constexpr float kPivotTol = 1e-6f;  // relative pivot below which the Gram is taken as singular

__device__ __forceinline__ int packed_up(int i, int c, int k) { return i * k - i * (i - 1) / 2 + (c - i); }

// Upper Cholesky factor (FP32) of the FP64 k x k matrix G, one CTA: G = R^T R,
// R written row-major with zeros below the diagonal.  The upper triangle
// lives packed in shared memory (k (k + 1) / 2 floats).
__global__ void __launch_bounds__(kCholThreads) chol_kernel(const double* __restrict__ G, int k,
                                                            float* __restrict__ R, int* fail) {
  if (*(volatile int*)fail) return;
  extern __shared__ float A[];
  __shared__ float piv_s;
  __shared__ int bad_s;
  const int tid = threadIdx.x;
  for (int e = tid; e < k * k; e += kCholThreads) {
    const int i = e / k, c = e % k;
    if (c >= i) A[packed_up(i, c, k)] = (float)G[e];
  }
  if (tid == 0) bad_s = 0;
  __syncthreads();
  for (int j = 0; j < k; ++j) {
    if (tid == 0) {
      const float d = A[packed_up(j, j, k)];
      const float g = (float)G[(int64_t)j * k + j];
      if (!(d > kPivotTol * g) || !(g > 0.f)) {
        bad_s = 1;
        piv_s = 1.f;
      } else {
        const float r = sqrtf(d);
        A[packed_up(j, j, k)] = r;
        piv_s = 1.f / r;
      }
    }
    __syncthreads();
    if (bad_s) break;  // uniform
    const float inv = piv_s;
    const int row = packed_up(j, j, k);
    for (int c = j + 1 + tid; c < k; c += kCholThreads) A[row + (c - j)] *= inv;
    __syncthreads();
    // trailing upper triangle: A[i][c] -= R[j][i] R[j][c], j < i <= c; warps
    // take rows, lanes consecutive columns
    {
      const int warp = tid >> 5, lane = tid & 31;
      for (int ii = j + 1 + warp; ii < k; ii += kCholThreads / 32) {
        const float rji = A[row + (ii - j)];
        float* arow = A + packed_up(ii, ii, k) - ii;  // arow[c] = A[ii][c]
        for (int cc = ii + lane; cc < k; cc += 32) arow[cc] -= rji * A[row + (cc - j)];
      }
    }
    __syncthreads();
  }
  if (bad_s) {
    if (tid == 0) atomicExch(fail, 1);
    return;
  }
  for (int e = tid; e < k * k; e += kCholThreads) {
    const int i = e / k, c = e % k;
    R[e] = c >= i ? A[packed_up(i, c, k)] : 0.f;
  }
}

// Rinv = R^-1 (upper triangular, FP32), one thread per column: back
// substitution of R x = e_c.  Zeros once the flag is set.
__global__ void tri_inv_kernel(const float* __restrict__ R, int k, float* __restrict__ Rinv, const int* fail) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= k) return;
  if (*(volatile const int*)fail) {  // zeros: the products that follow stay finite
    for (int i = 0; i < k; ++i) Rinv[(int64_t)i * k + c] = 0.f;
    return;
  }
  for (int i = k - 1; i > c; --i) Rinv[(int64_t)i * k + c] = 0.f;
  const float xc = 1.f / __ldg(R + (int64_t)c * k + c);
  Rinv[(int64_t)c * k + c] = xc;
  for (int i = c - 1; i >= 0; --i) {
    float s = 0.f;
    for (int l = i + 1; l <= c; ++l) s = fmaf(__ldg(R + (int64_t)i * k + l), Rinv[(int64_t)l * k + c], s);
    Rinv[(int64_t)i * k + c] = -s / __ldg(R + (int64_t)i * k + i);
  }
}

// R = R2 R1 in FP64 (both upper triangular), one CTA per column.
__global__ void rmul_kernel(const float* __restrict__ R2, const float* __restrict__ R1, int k, double* __restrict__ R,
                            const int* fail) {
  if (*(volatile const int*)fail) return;
  const int c = blockIdx.x;
  for (int i = threadIdx.x; i < k; i += blockDim.x) {
    double s = 0.0;
    if (i <= c)
      for (int l = i; l <= c; ++l) s += (double)R2[(int64_t)i * k + l] * (double)R1[(int64_t)l * k + c];
    R[(int64_t)i * k + c] = s;
  }
}

}  // namespace

size_t cholqr_smem_bytes(int k) { return (size_t)k * (k + 1) / 2 * sizeof(float); }

void launch_chol(Launcher& L, const double* G, int k, float* R, int* fail) {
  const size_t smem = cholqr_smem_bytes(k);
  cudaFuncSetAttribute(chol_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  chol_kernel<<<1, kCholThreads, smem, L.stream>>>(G, k, R, fail);
  L.count(1);
}

void launch_tri_inv(Launcher& L, const float* R, int k, float* Rinv, const int* fail) {
  tri_inv_kernel<<<(k + 63) / 64, 64, 0, L.stream>>>(R, k, Rinv, fail);
  L.count(1);
}

void launch_rmul(Launcher& L, const float* R2, const float* R1, int k, double* R, const int* fail) {
  rmul_kernel<<<k, 128, 0, L.stream>>>(R2, R1, k, R, fail);
  L.count(1);
}

}  // namespace lspca
