// K3: the operation on the small k x k matrix (table footnote of Sec. III):
//   H = F F^T,  H = W Lambda W^T (descending),  D = Lambda^1/2,  V = F^T W D^-1,
// followed by the sign rule (largest-|.| entry of each column positive, ties to
// the lowest index) and the rank rule (lambda_i <= max(m, n) 2^-52 lambda_1 ->
// column dropped, sigma_i = 0).
//
// GB300 executes FP64 at a small fraction of its FP32 rate, so the eigensolve
// is split into an FP32 cyclic Jacobi on one CTA (the seed) and FP64 iterative
// refinement of the whole eigenvector matrix built from k x k FP64 products
// spread over many CTAs (Ogita & Aishima, "Iterative refinement for symmetric
// eigenvalue decomposition", Japan J. Indust. Appl. Math. 35, 2018: one step
// forms R = I - X^T X, S = X^T H X, lambda_i = s_ii / (1 - r_ii),
// E_ij = (s_ij + lambda_j r_ij) / (lambda_j - lambda_i) for separated pairs,
// r_ij / 2 inside clusters, and updates X <- X + X E; it converges
// quadratically; the cluster test here is per pair, see refine_e_kernel).
// H, the refinement and V = F^T W D^-1 are FP64 throughout.
#include "common.cuh"
#include "kernels.h"

namespace lspca {

constexpr int kRefineIters = 3;
constexpr int kJacobiMaxSweeps = 16;
constexpr int kJacobiThreads = 1024;

size_t small_ws_bytes(int k, int64_t n, int* h_splits) {
  int hs = (int)((n + 511) / 512);
  if (hs < 1) hs = 1;
  if (hs > 64) hs = 64;
  if (h_splits) *h_splits = hs;
  const size_t kk = (size_t)k * k;
  size_t b = 0;
  b += (size_t)hs * kk * 8;            // Hpart
  b += kk * 8;                          // H
  b += kk * 4 * 2;                      // h32, w32
  b += kk * 8 * 6;                      // Xa Xb Rm T S E
  b += (size_t)k * 8 + 64;              // lam, scal
  b += (size_t)n * k * 8;               // Vd
  b += 64;                              // sweeps
  return b + 16 * 256;                  // alignment slack
}

static char* align256(char* p) { return (char*)(((uintptr_t)p + 255) & ~(uintptr_t)255); }

void carve_small_ws(SmallWs& w, void* base, int k, int64_t n) {
  int hs;
  small_ws_bytes(k, n, &hs);
  w.h_splits = hs;
  const size_t kk = (size_t)k * k;
  char* p = align256((char*)base);
  auto take = [&](size_t bytes) { char* r = p; p = align256(p + bytes); return r; };
  w.Hpart = (double*)take((size_t)hs * kk * 8);
  w.H = (double*)take(kk * 8);
  w.h32 = (float*)take(kk * 4);
  w.w32 = (float*)take(kk * 4);
  w.Xa = (double*)take(kk * 8);
  w.Xb = (double*)take(kk * 8);
  w.Rm = (double*)take(kk * 8);
  w.T = (double*)take(kk * 8);
  w.S = (double*)take(kk * 8);
  w.E = (double*)take(kk * 8);
  w.lam = (double*)take((size_t)k * 8);
  w.scal = (double*)take(64);
  w.Vd = (double*)take((size_t)n * k * 8);
  w.sweeps = (int32_t*)take(64);
}

// Round-robin ("circle") pairing: k2 players (k2 even), round t, pair r.
__device__ __forceinline__ void rr_pair(int k2, int t, int r, int& p, int& q) {
  const int K1 = k2 - 1;
  auto player = [&](int slot) { return slot == 0 ? 0 : 1 + ((slot - 1 + t) % K1); };
  const int a = player(r), b = player(k2 - 1 - r);
  p = a < b ? a : b;
  q = a < b ? b : a;
}

// FP32 cyclic Jacobi on H / scale.  One CTA of 1024 threads; H and W live in
// shared memory for k <= 128 and in the global scratch otherwise.  Rotations of
// one round act on disjoint index pairs: rows first, then columns (A <- J^T A J)
// and the columns of W (W <- W J).
__global__ void __launch_bounds__(kJacobiThreads) jacobi32_kernel(const double* __restrict__ H, int k, float* hg,
                                                                  float* wg, double* Xout, double* lam_out,
                                                                  int32_t* sweeps_out, int* status) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ float cs[128], sn[128];
  __shared__ int pp[128], qq[128];
  __shared__ int rotated;
  __shared__ float scale_s;
  const bool in_smem = k <= 128;
  float* h = in_smem ? reinterpret_cast<float*>(smem_raw) : hg;
  float* w = in_smem ? reinterpret_cast<float*>(smem_raw) + k * k : wg;
  const int tid = threadIdx.x;
  if (tid == 0) {
    double mx = 0.0;
    for (int i = 0; i < k; ++i) mx = fmax(mx, fabs(H[(int64_t)i * k + i]));
    scale_s = (float)(mx > 0.0 ? 1.0 / mx : 1.0);
  }
  __syncthreads();
  const double sc = (double)scale_s;
  for (int e = tid; e < k * k; e += kJacobiThreads) {
    h[e] = (float)(H[e] * sc);
    w[e] = (e / k == e % k) ? 1.f : 0.f;
  }
  const int k2 = (k % 2) ? k + 1 : k;
  const int npairs = k2 / 2;
  int sweep = 0;
  for (sweep = 0; sweep < kJacobiMaxSweeps; ++sweep) {
    if (tid == 0) rotated = 0;
    __syncthreads();
    for (int t = 0; t < k2 - 1; ++t) {
      if (tid < npairs) {
        int p, q;
        rr_pair(k2, t, tid, p, q);
        float c = 1.f, s = 0.f;
        if (q < k) {
          const float app = h[p * k + p], aqq = h[q * k + q], apq = h[p * k + q];
          // relative criterion, with a floor at FP32 rounding noise of the
          // scaled matrix (max diagonal = 1): below it the FP64 refinement takes over
          const float thr = fmaxf(1e-7f * sqrtf(fabsf(app * aqq)), 1e-6f);
          if (fabsf(apq) > thr) {
            const float tau = (aqq - app) / (2.f * apq);
            float tt = (tau >= 0.f ? 1.f : -1.f) / (fabsf(tau) + sqrtf(1.f + tau * tau));
            c = rsqrtf(1.f + tt * tt);
            s = tt * c;
            rotated = 1;
          }
        } else {
          q = p;  // dummy partner of an odd k: no rotation
        }
        cs[tid] = c;
        sn[tid] = s;
        pp[tid] = p;
        qq[tid] = q;
      }
      __syncthreads();
      // rows p, q of h
      for (int e = tid; e < npairs * k; e += kJacobiThreads) {
        const int r = e / k, j = e % k;
        const int p = pp[r], q = qq[r];
        if (p == q || sn[r] == 0.f) continue;
        const float c = cs[r], s = sn[r];
        const float hp = h[p * k + j], hq = h[q * k + j];
        h[p * k + j] = c * hp - s * hq;
        h[q * k + j] = s * hp + c * hq;
      }
      __syncthreads();
      // columns p, q of h and of w
      for (int e = tid; e < npairs * k; e += kJacobiThreads) {
        const int r = e / k, i = e % k;
        const int p = pp[r], q = qq[r];
        if (p == q || sn[r] == 0.f) continue;
        const float c = cs[r], s = sn[r];
        const float hp = h[i * k + p], hq = h[i * k + q];
        h[i * k + p] = c * hp - s * hq;
        h[i * k + q] = s * hp + c * hq;
        const float wp = w[i * k + p], wq = w[i * k + q];
        w[i * k + p] = c * wp - s * wq;
        w[i * k + q] = s * wp + c * wq;
      }
      __syncthreads();
      if (tid < npairs) {
        const int p = pp[tid], q = qq[tid];
        if (p != q && sn[tid] != 0.f) {
          h[p * k + q] = 0.f;
          h[q * k + p] = 0.f;
        }
      }
      __syncthreads();
    }
    if (!rotated) break;
  }
  for (int e = tid; e < k * k; e += kJacobiThreads) Xout[e] = (double)w[e];
  for (int i = tid; i < k; i += kJacobiThreads) lam_out[i] = (double)h[i * k + i] / sc;
  if (tid == 0) *sweeps_out = sweep < kJacobiMaxSweeps ? sweep + 1 : sweep;
}

// Block-wide FP64 sum (blockDim.x multiple of 32, <= 1024).
__device__ double block_sum(double v, double* red) {
  v = warp_sum(v);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) red[wid] = v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x == 0) {
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) s += red[i];
    red[32] = s;
  }
  __syncthreads();
  return red[32];
}

// One refinement step's small part: lambda_i = S_ii / (X^T X)_ii and the
// correction E (Rm = X^T X, R = I - Rm).  A pair (i, j) takes the first-order
// correction (s_ij + lambda_j r_ij) / (lambda_j - lambda_i) when that is a
// small rotation (|E_ij| <= 1/2) and the gap is above FP64 noise of H;
// otherwise it is treated as a cluster and only re-orthogonalised (r_ij / 2).
// The per-pair test replaces the method's global cluster threshold, which
// (evaluated with Frobenius norms) would leave close but well-coupled pairs
// unresolved; the iteration still converges quadratically for resolved pairs.
__global__ void refine_e_kernel(const double* __restrict__ H, const double* __restrict__ Rm,
                                const double* __restrict__ S, int k, double* __restrict__ E, double* lam) {
  __shared__ double red[33];
  __shared__ double lam_s[256];
  const int tid = threadIdx.x;
  for (int i = tid; i < k; i += blockDim.x) lam_s[i] = S[(int64_t)i * k + i] / Rm[(int64_t)i * k + i];
  double hh = 0.0;
  for (int e = tid; e < k * k; e += blockDim.x) hh += H[e] * H[e];
  hh = block_sum(hh, red);
  const double noise = 64.0 * 0x1p-52 * sqrt(hh);
  for (int e = tid; e < k * k; e += blockDim.x) {
    const int i = e / k, j = e % k;
    const double r = (i == j ? 1.0 : 0.0) - Rm[e];
    double v = 0.5 * r;
    if (i != j) {
      const double gap = lam_s[j] - lam_s[i];
      const double num = S[e] + lam_s[j] * r;
      if (fabs(gap) > noise && fabs(num) <= 0.5 * fabs(gap)) v = num / gap;
    }
    E[e] = v;
  }
  for (int i = tid; i < k; i += blockDim.x) lam[i] = lam_s[i];
}

// C = A + A E (k x k, FP64), one thread per output.
__global__ void add_ae_kernel(const double* __restrict__ A, const double* __restrict__ AE, int k, double* __restrict__ C) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e < k * k) C[e] = A[e] + AE[e];
}

// Sort eigenpairs by descending lambda (stable), apply the rank rule, write
// sigma (device output) and the permuted, D^-1-scaled eigenvector matrix
// Wd[:, r] = W[:, order_r] / sigma_r (zero for dropped columns).
__global__ void sort_rank_kernel(const double* __restrict__ lam, const double* __restrict__ W, int k, int64_t m,
                                 int64_t n, double* __restrict__ Wd, double* __restrict__ sigma, int32_t* rank,
                                 double* scal) {
  __shared__ int dest[256];
  __shared__ double lmax_s;
  __shared__ int rank_s;
  const int tid = threadIdx.x;
  for (int i = tid; i < k; i += blockDim.x) {
    const double li = lam[i];
    int pos = 0;
    for (int j = 0; j < k; ++j) {
      const double lj = lam[j];
      pos += (lj > li) || (lj == li && j < i);
    }
    dest[i] = pos;
  }
  __syncthreads();
  if (tid == 0) {
    double mx = 0.0;
    for (int i = 0; i < k; ++i) mx = fmax(mx, lam[i]);
    lmax_s = mx;
    rank_s = 0;
  }
  __syncthreads();
  const double tol = (double)(m > n ? m : n) * 0x1p-52 * lmax_s;
  for (int i = tid; i < k; i += blockDim.x) {
    const int r = dest[i];
    const bool keep = lam[i] > tol && lmax_s > 0.0;
    const double s = keep ? sqrt(lam[i]) : 0.0;
    if (sigma) sigma[r] = s;
    scal[8 + r] = s;
    if (keep) atomicAdd(&rank_s, 1);
    for (int row = 0; row < k; ++row) Wd[(int64_t)row * k + r] = keep ? W[(int64_t)row * k + i] / s : 0.0;
  }
  __syncthreads();
  if (tid == 0 && rank) *rank = rank_s;
  if (tid == 0) scal[0] = (double)rank_s;
}

// Sign rule and FP32 output: one block per column of Vd (n x k FP64).
template <typename VT>
__global__ void finalize_v_kernel(const double* __restrict__ Vd, int64_t n, int k, VT* __restrict__ V) {
  __shared__ double bv[32];
  __shared__ int64_t bi[32];
  __shared__ double sgn_s;
  const int c = blockIdx.x;
  double best = -1.0;
  int64_t besti = 0;
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
    const double a = fabs(Vd[i * k + c]);
    if (a > best) { best = a; besti = i; }
  }
  // warp argmax, ties to the lowest index
  for (int o = 16; o > 0; o >>= 1) {
    const double ob = __shfl_xor_sync(0xffffffffu, best, o);
    const int64_t oi = __shfl_xor_sync(0xffffffffu, besti, o);
    if (ob > best || (ob == best && oi < besti)) { best = ob; besti = oi; }
  }
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) { bv[wid] = best; bi[wid] = besti; }
  __syncthreads();
  if (threadIdx.x == 0) {
    double b = -1.0;
    int64_t ix = 0;
    for (int wdx = 0; wdx < (int)(blockDim.x >> 5); ++wdx)
      if (bv[wdx] > b || (bv[wdx] == b && bi[wdx] < ix)) { b = bv[wdx]; ix = bi[wdx]; }
    sgn_s = (Vd[ix * k + c] < 0.0) ? -1.0 : 1.0;
  }
  __syncthreads();
  const double sg = sgn_s;
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) V[i * k + c] = (VT)(sg * Vd[i * k + c]);
}

static void dgemm(Launcher& L, int64_t M, int64_t N, int64_t K, const double* A, int64_t lda, bool at, const double* B,
                  int64_t ldb, bool bt, double* C, int64_t ldc) {
  launch_gemm_simt(L, M, N, K, A, LSPCA_F64, lda, at, B, LSPCA_F64, ldb, bt, C, true, ldc, 0, 1, true, true);
}

void launch_decompose(Launcher& L, SmallWs& w, const double* F, int k, int64_t n, int64_t m, bool v_f64, void* V,
                      double* sigma, int32_t* rank, int* status) {
  const int64_t kk = (int64_t)k * k;
  // H = F F^T, split over n, reduced in fixed order.
  launch_gemm_simt(L, k, k, n, F, LSPCA_F64, n, false, F, LSPCA_F64, n, true, w.Hpart, true, k, kk, w.h_splits, true,
                   true);
  launch_reduce_splits(L, w.Hpart, w.h_splits, kk, kk, w.H);
  // FP32 Jacobi seed.
  const size_t jsmem = (k <= 128) ? (size_t)2 * kk * sizeof(float) : 0;
  cudaFuncSetAttribute(jacobi32_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)(jsmem ? jsmem : 0));
  jacobi32_kernel<<<1, kJacobiThreads, jsmem, L.stream>>>(w.H, k, w.h32, w.w32, w.Xa, w.lam, w.sweeps, status);
  L.count(1);
  // FP64 refinement.
  double* X = w.Xa;
  double* Xn = w.Xb;
  for (int it = 0; it <= kRefineIters; ++it) {
    dgemm(L, k, k, k, X, k, true, X, k, false, w.Rm, k);    // X^T X
    dgemm(L, k, k, k, w.H, k, false, X, k, false, w.T, k);  // H X
    dgemm(L, k, k, k, X, k, true, w.T, k, false, w.S, k);   // X^T H X
    refine_e_kernel<<<1, 1024, 0, L.stream>>>(w.H, w.Rm, w.S, k, w.E, w.lam);
    L.count(1);
    if (it == kRefineIters) break;  // last pass only refreshes lambda
    dgemm(L, k, k, k, X, k, false, w.E, k, false, w.T, k);  // X E
    add_ae_kernel<<<(int)((kk + 255) / 256), 256, 0, L.stream>>>(X, w.T, k, Xn);
    L.count(1);
    double* t = X;
    X = Xn;
    Xn = t;
  }
  // order, rank rule, D^-1 folded into the eigenvector matrix
  sort_rank_kernel<<<1, 256, 0, L.stream>>>(w.lam, X, k, m, n, w.E, sigma, rank, w.scal);
  L.count(1);
  // V = F^T (W D^-1)  (n x k)
  launch_gemm_simt(L, n, k, k, F, LSPCA_F64, n, true, w.E, LSPCA_F64, k, false, w.Vd, true, k, 0, 1, true, true);
  if (v_f64)
    finalize_v_kernel<double><<<k, 256, 0, L.stream>>>(w.Vd, n, k, (double*)V);
  else
    finalize_v_kernel<float><<<k, 256, 0, L.stream>>>(w.Vd, n, k, (float*)V);
  L.count(1);
}

}  // namespace lspca
