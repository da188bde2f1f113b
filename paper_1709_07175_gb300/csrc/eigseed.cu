// FP32 seed of the symmetric eigensolve of the k x k step (one CTA).
//
// The FP64 refinement that follows (small.cu) needs eigenvectors accurate to
// well under a radian per pair; a standard dense symmetric route gives them in
// O(k^3) flops with O(k) synchronisations:
//   1. Householder tridiagonalisation  H = Q T Q^T  (reflectors kept in the
//      lower triangle, as in LAPACK's sytrd);
//   2. eigenvalues of T by bisection on Sturm counts, one thread per
//      eigenvalue, 30 halvings of the Gershgorin interval (FP32 resolution);
//   3. eigenvectors of T by two steps of inverse iteration with an LDL^T solve
//      of T - lambda I; eigenvalues closer than 1e-5 ||T|| form a cluster whose
//      vectors are computed in order by one thread and Gram-Schmidt
//      orthogonalised against (up to 32 of) the cluster's earlier vectors, as
//      LAPACK's stein does (which uses 1e-3 ||T||: pairs between the two
//      thresholds come out non-orthogonal by at most ~1e-2 here, well inside
//      what the FP64 refinement corrects);
//   4. back-transformation W = Q Z.
// H is scaled by 1 / max|H_ii| first.  Matrices live in shared memory for
// k <= 128 and in a global scratch otherwise; Householder vectors are copied
// to a contiguous vector before use (a column of the row-major matrix would
// bank-conflict on every read).
#include "common.cuh"
#include "kernels.h"

namespace lspca {

constexpr int kSeedThreads = 512;

__device__ __forceinline__ float block_sum_f(float v, float* red) {
  v = warp_sumf(v);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) red[wid] = v;
  __syncthreads();
  if (threadIdx.x < 32) {
    float s = (threadIdx.x < (int)(blockDim.x >> 5)) ? red[threadIdx.x] : 0.f;
    s = warp_sumf(s);
    if (threadIdx.x == 0) red[32] = s;
  }
  __syncthreads();
  return red[32];
}

// Number of eigenvalues of T (d, e) smaller than x (Sturm count).
__device__ __forceinline__ int sturm_count(const float* d, const float* e2, int k, float x, float pivmin) {
  int c = 0;
  float q = d[0] - x;
  if (fabsf(q) < pivmin) q = -pivmin;
  c += q < 0.f;
  for (int i = 1; i < k; ++i) {
    q = d[i] - x - __fdividef(e2[i - 1], q);
    if (fabsf(q) < pivmin) q = -pivmin;
    c += q < 0.f;
  }
  return c;
}

// One inverse-iteration solve (T - lam I) z <- z with the LDL^T factorisation
// (no pivoting; tiny pivots replaced by -pivmin), then normalisation.
// q is per-thread scratch of length k.
__device__ __forceinline__ void inv_iter(const float* d, const float* e, int k, float lam, float pivmin, float* z, float* q,
                         int zstride, int qstride) {
  // factor: q_0 = d_0 - lam, q_i = d_i - lam - e_{i-1}^2 / q_{i-1}; L_i = e_{i-1} / q_{i-1}
  float qi = d[0] - lam;
  if (fabsf(qi) < pivmin) qi = -pivmin;
  q[0] = qi;
  for (int i = 1; i < k; ++i) {
    qi = d[i] - lam - __fdividef(e[i - 1] * e[i - 1], qi);
    if (fabsf(qi) < pivmin) qi = -pivmin;
    q[i * qstride] = qi;
  }
  // forward: L y = z  (L unit lower bidiagonal, L_i = e_{i-1}/q_{i-1})
  for (int i = 1; i < k; ++i) z[i * zstride] -= __fdividef(e[i - 1], q[(i - 1) * qstride]) * z[(i - 1) * zstride];
  // diagonal and backward: D L^T x = y
  z[(k - 1) * zstride] = __fdividef(z[(k - 1) * zstride], q[(k - 1) * qstride]);
  for (int i = k - 2; i >= 0; --i) {
    const float rq = __fdividef(1.f, q[i * qstride]);
    z[i * zstride] = z[i * zstride] * rq - (e[i] * rq) * z[(i + 1) * zstride];
  }
  float nrm = 0.f;
  for (int i = 0; i < k; ++i) nrm = fmaf(z[i * zstride], z[i * zstride], nrm);
  if (!(nrm > 0.f) || !isfinite(nrm)) {
    // overflow or a zero solve: fall back to a coordinate vector
    for (int i = 0; i < k; ++i) z[i * zstride] = 0.f;
    z[0] = 1.f;
    return;
  }
  const float inv = rsqrtf(nrm);
  for (int i = 0; i < k; ++i) z[i * zstride] *= inv;
}

__global__ void __launch_bounds__(kSeedThreads, 1) eig_seed_kernel(const double* __restrict__ H, int k, float* gA,
                                                                float* gZ, float* gQ, double* __restrict__ Xout,
                                                                double* __restrict__ lam_out, double* scal,
                                                                int32_t* nclusters) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ float red[33];
  __shared__ float dv[256], ev[256], e2v[256], betav[256], wl[256], pv[256], lamv[256], vv_s[256];
  __shared__ float gpart[512];
  __shared__ float coef[4];
  __shared__ int clstart[257];
  const bool sm = k <= 128;
  float* A = sm ? reinterpret_cast<float*>(smem_raw) : gA;         // k x k row-major
  float* Z = sm ? reinterpret_cast<float*>(smem_raw) + k * k : gZ;  // k x k, column j = eigenvector j
  float* Qs = sm ? reinterpret_cast<float*>(smem_raw) + 2 * k * k : gQ;  // inverse-iteration scratch, one row per cluster
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = kSeedThreads / 32;

  // scale and load; ||H||_F for the refinement's noise floor
  __shared__ double hmax_s;
  if (tid == 0) {
    double mx = 0.0;
    for (int i = 0; i < k; ++i) mx = fmax(mx, fabs(H[(int64_t)i * k + i]));
    hmax_s = mx > 0.0 ? mx : 1.0;
  }
  __syncthreads();
  const double sc = 1.0 / hmax_s;
  double hf = 0.0;
  for (int e = tid; e < k * k; e += kSeedThreads) {
    const double h = H[e];
    hf += h * h;
    A[e] = (float)(h * sc);
  }
  hf = warp_sum(hf);
  {
    __shared__ double redd[32];
    if (lane == 0) redd[warp] = hf;
    __syncthreads();
    if (tid == 0) {
      double s = 0.0;
      for (int i = 0; i < nw; ++i) s += redd[i];
      scal[1] = sqrt(s);
    }
  }
  __syncthreads();

  // ---- 1. tridiagonalisation
  for (int j = 0; j + 2 < k; ++j) {
    const int n1 = k - j - 1;
    float part = 0.f;
    for (int i = j + 2 + tid; i < k; i += kSeedThreads) {
      const float x = A[i * k + j];
      part = fmaf(x, x, part);
    }
    const float sig = block_sum_f(part, red);
    if (tid == 0) {
      const float x0 = A[(j + 1) * k + j];
      const float nrm = sqrtf(x0 * x0 + sig);
      float alpha = 0.f, beta = 0.f;
      if (nrm > 0.f) {
        alpha = x0 >= 0.f ? -nrm : nrm;
        const float v0 = x0 - alpha;
        const float vv = v0 * v0 + sig;
        beta = vv > 0.f ? 2.f / vv : 0.f;
        A[(j + 1) * k + j] = v0;
      }
      dv[j] = A[j * k + j];
      ev[j] = (nrm > 0.f) ? alpha : x0;
      betav[j] = beta;
    }
    __syncthreads();
    const float beta = betav[j];
    if (beta != 0.f) {
      // v (column j below the diagonal) into a contiguous vector: the column is
      // strided by k in SMEM and would bank-conflict on every read
      for (int r = tid; r < n1; r += kSeedThreads) vv_s[r] = A[(j + 1 + r) * k + j];
      __syncthreads();
      // p = beta A' v, A' = A[j+1:, j+1:]; one warp per row
      for (int r = warp; r < n1; r += nw) {
        const float* row = A + (j + 1 + r) * k + (j + 1);
        float acc = 0.f;
        for (int l = lane; l < n1; l += 32) acc = fmaf(row[l], vv_s[l], acc);
        acc = warp_sumf(acc);
        if (lane == 0) pv[r] = beta * acc;
      }
      __syncthreads();
      float pt = 0.f;
      for (int r = tid; r < n1; r += kSeedThreads) pt = fmaf(pv[r], vv_s[r], pt);
      const float ptv = block_sum_f(pt, red);
      const float K = 0.5f * beta * ptv;
      for (int r = tid; r < n1; r += kSeedThreads) wl[r] = pv[r] - K * vv_s[r];
      __syncthreads();
      for (int r = warp; r < n1; r += nw) {
        const float vr = vv_s[r], wr = wl[r];
        float* row = A + (j + 1 + r) * k + (j + 1);
        for (int c = lane; c < n1; c += 32) row[c] -= vr * wl[c] + wr * vv_s[c];
      }
      __syncthreads();
    }
  }
  if (tid == 0) {
    if (k >= 2) {
      dv[k - 2] = A[(k - 2) * k + (k - 2)];
      ev[k - 2] = A[(k - 1) * k + (k - 2)];
    }
    dv[k - 1] = A[(k - 1) * k + (k - 1)];
    if (k >= 2) betav[k - 2] = 0.f;
    betav[k - 1] = 0.f;
  }
  __syncthreads();
  for (int i = tid; i < k; i += kSeedThreads) e2v[i] = (i + 1 < k) ? ev[i] * ev[i] : 0.f;

  // Gershgorin interval, ||T||, pivmin
  if (tid == 0) {
    float gl = 1e30f, gu = -1e30f, tn = 0.f;
    for (int i = 0; i < k; ++i) {
      const float off = (i > 0 ? fabsf(ev[i - 1]) : 0.f) + (i + 1 < k ? fabsf(ev[i]) : 0.f);
      gl = fminf(gl, dv[i] - off);
      gu = fmaxf(gu, dv[i] + off);
      tn = fmaxf(tn, fabsf(dv[i]) + off);
    }
    const float pad = 2.f * 1.2e-7f * tn + 1e-30f;
    coef[0] = gl - pad;
    coef[1] = gu + pad;
    coef[2] = tn;
    coef[3] = fmaxf(1e-30f, 1.2e-7f * 1e-6f * tn);  // pivmin
  }
  __syncthreads();
  const float tnorm = coef[2], pivmin = coef[3];

  // ---- 2. eigenvalues by bisection (one thread per eigenvalue, ascending index)
  for (int idx = tid; idx < k; idx += kSeedThreads) {
    float lo = coef[0], hi = coef[1];
#pragma unroll 1
    for (int it = 0; it < 30; ++it) {
      const float mid = 0.5f * (lo + hi);
      if (sturm_count(dv, e2v, k, mid, pivmin) > idx) hi = mid;
      else lo = mid;
    }
    lamv[idx] = 0.5f * (lo + hi);
  }
  __syncthreads();

  // ---- 3. eigenvectors of T: clusters of close eigenvalues, inverse iteration
  if (tid == 0) {
    int nc = 0;
    for (int i = 0; i < k; ++i)
      if (i == 0 || lamv[i] - lamv[i - 1] > 1e-5f * tnorm) clstart[nc++] = i;
    clstart[nc] = k;
    clstart[256] = nc;
    *nclusters = nc;
  }
  __syncthreads();
  const int ncl = clstart[256];
  for (int cl = tid; cl < ncl; cl += kSeedThreads) {
    const int i0 = clstart[cl], i1 = clstart[cl + 1];
    float* q = Qs + cl;  // element i at q[i * k]: the threads of a warp (clusters) hit consecutive banks
    for (int i = i0; i < i1; ++i) {
      // deterministic start vector, then two solves with Gram-Schmidt against
      // the cluster's earlier vectors after each
      for (int r = 0; r < k; ++r) Z[r * k + i] = 1.f + 0.5f * __sinf(0.7f * (float)(r + 3 * i) + 0.3f);
      const float lam = lamv[i];
      for (int rep = 0; rep < 2; ++rep) {
        inv_iter(dv, ev, k, lam, pivmin, Z + i, q, k, k);
        for (int pj = (i - 32 > i0 ? i - 32 : i0); pj < i; ++pj) {
          float dot = 0.f;
          for (int r = 0; r < k; ++r) dot = fmaf(Z[r * k + pj], Z[r * k + i], dot);
          float nrm = 0.f;
          for (int r = 0; r < k; ++r) {
            Z[r * k + i] -= dot * Z[r * k + pj];
            nrm = fmaf(Z[r * k + i], Z[r * k + i], nrm);
          }
          const float inv = nrm > 0.f ? rsqrtf(nrm) : 1.f;
          for (int r = 0; r < k; ++r) Z[r * k + i] *= inv;
        }
      }
    }
  }
  __syncthreads();

  // ---- 4. back-transformation: Z <- H_0 H_1 ... H_{k-3} Z
  for (int j = k - 3; j >= 0; --j) {
    const float beta = betav[j];
    if (beta == 0.f) continue;
    const int n1 = k - j - 1;
    for (int r = tid; r < n1; r += kSeedThreads) vv_s[r] = A[(j + 1 + r) * k + j];
    __syncthreads();
    // w_c = beta v^T Z[j+1:, c]: thread = (row group g, column c), consecutive
    // threads take consecutive columns (conflict-free), partials summed via SMEM
    {
      const int groups = kSeedThreads / k;  // 4 for k = 128, 2 for k = 256
      for (int t = tid; t < groups * k; t += kSeedThreads) {
        const int c = t % k, g = t / k;
        float acc = 0.f;
        for (int r = g; r < n1; r += groups) acc = fmaf(vv_s[r], Z[(j + 1 + r) * k + c], acc);
        gpart[g * k + c] = acc;
      }
      __syncthreads();
      for (int c = tid; c < k; c += kSeedThreads) {
        float acc = 0.f;
        for (int g = 0; g < groups; ++g) acc += gpart[g * k + c];
        wl[c] = beta * acc;
      }
    }
    __syncthreads();
    for (int r = warp; r < n1; r += nw) {
      const float vr = vv_s[r];
      float* row = Z + (j + 1 + r) * k;
      for (int c = lane; c < k; c += 32) row[c] -= vr * wl[c];
    }
    __syncthreads();
  }
  for (int e = tid; e < k * k; e += kSeedThreads) Xout[e] = (double)Z[e];
  for (int i = tid; i < k; i += kSeedThreads) lam_out[i] = (double)lamv[i] * hmax_s;
}

size_t eig_seed_smem(int k) { return k <= 128 ? (size_t)3 * k * k * sizeof(float) : 0; }

void launch_eig_seed(Launcher& L, const double* H, int k, float* gA, float* gZ, float* gQ, double* Xout,
                     double* lam, double* scal, int32_t* nclusters) {
  const size_t shm = eig_seed_smem(k);
  cudaFuncSetAttribute(eig_seed_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm);
  eig_seed_kernel<<<1, kSeedThreads, shm, L.stream>>>(H, k, gA, gZ, gQ, Xout, lam, scal, nclusters);
  L.count(1);
}

}  // namespace lspca
