// K4: tall-skinny QR for the SPCA comparison path (Algorithms 1 and 3).
//
// Algorithm 3 keeps a running R with qr([R; U_s]) per slice.  On the GPU the
// same factor comes from a reduction tree: every block of 2k rows of U is
// factored by Householder reflections into a k x k R, then pairs of R factors
// are stacked and factored again until one R remains (R^T R = U^T U, rows of R
// determined up to sign).  Only R is kept (Q is never formed, as in Algorithm
// 3).  Each factorisation runs on one CTA with the 2k x k working matrix in
// shared memory (global scratch when it does not fit); FP64 for FP64 U, FP32
// otherwise.  F_s = R^-T F is then a forward substitution in FP64.
#include "common.cuh"
#include "kernels.h"

namespace lspca {

constexpr int kQrThreads = 512;
constexpr int kSmemLimit = 200 * 1024;

__host__ __device__ __forceinline__ int qr_rows(int k) { return 2 * k; }

template <typename Acc>
static bool qr_in_smem(int k) {
  return (size_t)qr_rows(k) * k * sizeof(Acc) + 4096 <= (size_t)kSmemLimit;
}

size_t tsqr_ws_bytes(int64_t m, int k) {
  const int B = qr_rows(k);
  const int64_t nb0 = (m + B - 1) / B;
  // two R stacks (ping-pong, FP64) + per-CTA global working matrices (FP64 bound)
  const size_t rstack = (size_t)nb0 * k * k * 8;
  const size_t work = (size_t)(nb0 < 4096 ? nb0 : 4096) * B * k * 8;
  return 2 * rstack + work + 1024;
}

// Factor one block.  Rows come from `src` (row-major, ld ksrc) rows [r0, r1),
// or, for a tree node, from two R factors stacked.  Writes the k x k upper
// triangular R (row-major, FP64) to `dst`.
template <typename Acc, typename SrcT>
__global__ void __launch_bounds__(kQrThreads) qr_block_kernel(const SrcT* __restrict__ src, int64_t m, int k,
                                                              int rows_per_block, const double* __restrict__ rin,
                                                              int nin, double* __restrict__ rout, Acc* gwork,
                                                              int use_smem, const int* run_if) {
  if (run_if && *(volatile const int*)run_if == 0) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ Acc beta_s, rjj_s;
  const int B = qr_rows(k);
  const int b = blockIdx.x;
  Acc* Wm = use_smem ? reinterpret_cast<Acc*>(smem_raw) : gwork + (size_t)b * B * k;  // column-major B x k
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31, nwarps = kQrThreads / 32;

  // load
  for (int e = tid; e < B * k; e += kQrThreads) {
    const int r = e / k, c = e % k;
    Acc v = Acc(0);
    if (rin == nullptr) {
      const int64_t gr = (int64_t)b * rows_per_block + r;
      if (r < rows_per_block && gr < m) v = (Acc)src[gr * k + c];
    } else {
      const int which = 2 * b + (r >= k ? 1 : 0);
      const int rr = r >= k ? r - k : r;
      if (which < nin) v = (Acc)rin[(size_t)which * k * k + (size_t)rr * k + c];
    }
    Wm[(size_t)c * B + r] = v;
  }
  __syncthreads();

  // Rows a reflector touches.  A leaf block is dense: rows j .. B-1.  A tree
  // node stacks two upper triangles, so reflector j has nonzeros only in row
  // j and rows k .. k + j (the rows of the first triangle below j are still
  // zero, those of the second below k + j too), and its update touches only
  // those rows.  Lane l of a warp takes the l-th, (l+32)-th, ... of them.
  const bool node = rin != nullptr;
  auto row_at = [&](int j, int t) { return node ? (t == 0 ? j : k + t - 1) : j + t; };
  auto row_count = [&](int j) { return node ? j + 2 : B - j; };
  for (int j = 0; j < k; ++j) {
    Acc* colj = Wm + (size_t)j * B;
    const int nr = row_count(j);
    if (warp == 0) {
      // the diagonal of the previous step lands now (the update there read
      // v's leading entry from the same place), saving a barrier
      if (lane == 0 && j > 0) Wm[(size_t)(j - 1) * B + (j - 1)] = rjj_s;
      Acc sq = Acc(0);
      for (int t = 1 + lane; t < nr; t += 32) {
        const Acc x = colj[row_at(j, t)];
        sq += x * x;
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) sq += __shfl_xor_sync(0xffffffffu, sq, o);
      if (lane == 0) {
        const Acc alpha = colj[j];
        const Acc nrm = sqrt(alpha * alpha + sq);
        if (nrm == Acc(0)) {
          beta_s = Acc(0);
          rjj_s = Acc(0);
        } else {
          const Acc sg = alpha >= Acc(0) ? Acc(1) : Acc(-1);
          const Acc v0 = alpha + sg * nrm;
          colj[j] = v0;
          beta_s = Acc(2) / (v0 * v0 + sq);
          rjj_s = -sg * nrm;
        }
      }
    }
    __syncthreads();
    const Acc beta = beta_s;
    if (beta != Acc(0)) {
      // trailing columns j+1 .. k-1, four at a time per warp (independent
      // load / reduction / update chains)
      for (int c0 = j + 1 + 4 * warp; c0 < k; c0 += 4 * nwarps) {
        Acc* cc[4];
        Acc ws[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          cc[q] = Wm + (size_t)(c0 + q < k ? c0 + q : c0) * B;
          ws[q] = Acc(0);
        }
        for (int t = lane; t < nr; t += 32) {
          const int r = row_at(j, t);
          const Acc v = colj[r];
#pragma unroll
          for (int q = 0; q < 4; ++q) ws[q] += v * cc[q][r];
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
          for (int q = 0; q < 4; ++q) ws[q] += __shfl_xor_sync(0xffffffffu, ws[q], o);
        }
        for (int t = lane; t < nr; t += 32) {
          const int r = row_at(j, t);
          const Acc v = colj[r];
#pragma unroll
          for (int q = 0; q < 4; ++q)
            if (c0 + q < k) cc[q][r] -= beta * ws[q] * v;
        }
      }
    }
    __syncthreads();
  }
  if (tid == 0) Wm[(size_t)(k - 1) * B + (k - 1)] = rjj_s;
  __syncthreads();
  double* R = rout + (size_t)b * k * k;
  for (int e = tid; e < k * k; e += kQrThreads) {
    const int i = e / k, c = e % k;
    R[e] = (c >= i) ? (double)Wm[(size_t)c * B + i] : 0.0;
  }
}

__global__ void copy_r_kernel(const double* __restrict__ src, double* __restrict__ dst, int n, const int* run_if) {
  if (run_if && *(volatile const int*)run_if == 0) return;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n; e += gridDim.x * blockDim.x) dst[e] = src[e];
}

template <typename Acc, typename SrcT>
static void tsqr_typed(Launcher& L, const SrcT* U, int64_t m, int k, void* ws, double* R, const int* run_if) {
  const int B = qr_rows(k);
  const int64_t nb0 = (m + B - 1) / B;
  char* p = (char*)ws;
  double* ra = (double*)p;
  double* rb = ra + (size_t)nb0 * k * k;
  Acc* gwork = (Acc*)(rb + (size_t)nb0 * k * k);
  const bool smem = qr_in_smem<Acc>(k);
  const size_t shm = smem ? (size_t)B * k * sizeof(Acc) : 0;
  cudaFuncSetAttribute(qr_block_kernel<Acc, SrcT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm);
  // level 0: 4096 blocks per launch at most (bounded global scratch)
  for (int64_t b0 = 0; b0 < nb0; b0 += 4096) {
    const int nb = (int)((nb0 - b0) < 4096 ? (nb0 - b0) : 4096);
    qr_block_kernel<Acc, SrcT><<<nb, kQrThreads, shm, L.stream>>>(U + b0 * B * k, m - b0 * B, k, B, nullptr, 0,
                                                                   ra + (size_t)b0 * k * k, gwork, smem ? 1 : 0,
                                                                   run_if);
    L.count(1);
  }
  int64_t nin = nb0;
  double* cur = ra;
  double* nxt = rb;
  while (nin > 1) {
    const int64_t nout = (nin + 1) / 2;
    qr_block_kernel<Acc, SrcT><<<(int)nout, kQrThreads, shm, L.stream>>>(U, 0, k, B, cur, (int)nin, nxt, gwork,
                                                                         smem ? 1 : 0, run_if);
    L.count(1);
    double* t = cur;
    cur = nxt;
    nxt = t;
    nin = nout;
  }
  copy_r_kernel<<<(k * k + 255) / 256, 256, 0, L.stream>>>(cur, R, k * k, run_if);
  L.count(1);
}

void launch_tsqr(Launcher& L, const void* U, bool u_f64, int64_t m, int k, void* ws, double* R, const int* run_if) {
  if (u_f64)
    tsqr_typed<double, double>(L, (const double*)U, m, k, ws, R, run_if);
  else
    tsqr_typed<float, float>(L, (const float*)U, m, k, ws, R, run_if);
}

// F <- R^-T F: forward substitution on R^T (lower triangular), one thread per
// column of F; R (k x k FP64) is read through the read-only cache, every lane
// of a warp reading the same entry.  A pivot below rtol times the largest
// |R_ii| marks a direction U does not resolve (U rank deficient to working
// precision): that row of the result is 0.  Dividing by such a pivot would
// blow F's own rounding error (relative u) up to u / rtol, so rtol sits near
// sqrt(u): 1e-4 for FP32 U, 1e-10 for FP64 U.
__global__ void trsm_rt_kernel(const double* __restrict__ R, int k, double* __restrict__ F, int64_t n, double rtol) {
  const int64_t col = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (col >= n) return;
  double dmax = 0.0;
  for (int i = 0; i < k; ++i) dmax = fmax(dmax, fabs(__ldg(R + i * k + i)));
  const double tol = rtol * dmax;
  for (int i = 0; i < k; ++i) {
    double s = F[(int64_t)i * n + col];
    for (int l = 0; l < i; ++l) s -= __ldg(R + l * k + i) * F[(int64_t)l * n + col];
    const double d = __ldg(R + i * k + i);
    F[(int64_t)i * n + col] = fabs(d) > tol ? s / d : 0.0;
  }
}

void launch_trsm_rt(Launcher& L, const double* R, int k, double* F, int64_t n, bool u_f64) {
  const int threads = 32;
  trsm_rt_kernel<<<(int)((n + threads - 1) / threads), threads, 0, L.stream>>>(R, k, F, n, u_f64 ? 1e-10 : 1e-4);
  L.count(1);
}

}  // namespace lspca
