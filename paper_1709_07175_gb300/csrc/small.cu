// K3: the operation on the small k x k matrix (table footnote of Sec. III):
//   H = F F^T,  H = W Lambda W^T (descending),  D = Lambda^1/2,  V = F^T W D^-1,
// followed by the sign rule (largest-|.| entry of each column positive, ties to
// the lowest index) and the rank rule (lambda_i <= max(m, n) 2^-52 lambda_1 ->
// column dropped, sigma_i = 0).
//
// GB300 executes FP64 at a small fraction of its FP32 rate, so the eigensolve
// is split into an FP32 seed (tridiagonalisation, bisection, inverse
// iteration, eigseed.cu) and FP64 iterative refinement of the whole
// eigenvector matrix built from k x k FP64 products spread over many CTAs;
// the seed runs in up to kSeedLevels levels, each on the tail block the
// level before left unresolved (Ogita & Aishima, "Iterative refinement for symmetric
// eigenvalue decomposition", Japan J. Indust. Appl. Math. 35, 2018: one step
// forms R = I - X^T X, S = X^T H X, lambda_i = s_ii / (1 - r_ii),
// E_ij = (s_ij + lambda_j r_ij) / (lambda_j - lambda_i) for separated pairs,
// r_ij / 2 inside clusters, and updates X <- X + X E; it converges
// quadratically; the cluster test here is per pair, see refine_e_kernel).
// H and the refinement are FP64; V = F^T W D^-1 is an FP64 product for an
// FP64 V and an FP32 product of the FP64 factors for an FP32 V.
#include "common.cuh"
#include "kernels.h"

namespace lspca {

constexpr int kRefineIters = 2;
constexpr int kVT = 64;  // V tile of vprod_kernel (rows and columns)

static size_t vaux_bytes(int k, int64_t n) {
  return (size_t)((n + kVT - 1) / kVT) * k * 8 + 256 + (size_t)k * 4 + 256 + 64;
}

size_t small_ws_bytes(int k, int64_t n, int* h_splits) {
  int hs = (int)((n + 511) / 512);
  if (hs < 1) hs = 1;
  if (hs > 64) hs = 64;
  if (h_splits) *h_splits = hs;
  const size_t kk = (size_t)k * k;
  size_t b = 0;
  b += (size_t)hs * kk * 8;            // Hpart
  b += oz_gram_ws_bytes(k, n);          // tensor-core H
  b += kk * 8;                          // H
  b += kk * 4 * 4;                      // seed scratch: reflectors, Z, pivots / Householder vectors, QR copy
  b += kk * 8 * 6;                      // Xa Xb Rm T S E
  b += (size_t)k * 8 + 64 + (size_t)k * 24;  // lam, scal (+ src, sd)
  b += (size_t)n * k * 8;               // Vd
  b += vaux_bytes(k, n);                // V column maxima, signs, counters
  b += 64;                              // sweeps
  b += 64;                              // seed level sizes
  b += (size_t)k * 4;                   // seed cluster ids
  b += (size_t)k * 4 * 5 + 64;          // seed scratch: d, e, e^2, beta, eigenvalues of T, scalars
  return b + 24 * 256;                  // alignment slack
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
  w.oz = take(oz_gram_ws_bytes(k, n));
  w.H = (double*)take(kk * 8);
  w.h32 = (float*)take(kk * 4);
  w.w32 = (float*)take(kk * 4);
  w.q32 = (float*)take(kk * 4);
  w.p32 = (float*)take(kk * 4);
  w.Xa = (double*)take(kk * 8);
  w.Xb = (double*)take(kk * 8);
  w.Rm = (double*)take(kk * 8);
  w.T = (double*)take(kk * 8);
  w.S = (double*)take(kk * 8);
  w.E = (double*)take(kk * 8);
  w.lam = (double*)take((size_t)k * 8);
  w.scal = (double*)take(64 + (size_t)k * 24);
  w.Vd = (double*)take((size_t)n * k * 8);
  w.vaux = take(vaux_bytes(k, n));
  w.sweeps = (int32_t*)take(64);
  w.lvl = (int32_t*)take(64);
  w.cid = (int32_t*)take((size_t)k * 4);
  w.tri = (float*)take((size_t)k * 4 * 5 + 64);
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

// lambda_i = S_ii / (X^T X)_ii (Rayleigh quotients of the current vectors).
// act (nullable): the seed level's block size; below 2 the level is idle and
// the kernel leaves its outputs as they are.
__global__ void rayleigh_kernel(const double* __restrict__ Rm, const double* __restrict__ S, int k, double* lam,
                                const int32_t* act) {
  pdl_wait();  // first, on every path: completion stays ordered along the chain
  if (act && *act < 2) return;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < k; i += gridDim.x * blockDim.x)
    lam[i] = S[(int64_t)i * k + i] / Rm[(int64_t)i * k + i];
}

// Clusters the refinement resolves by Rayleigh-Ritz: runs of equal cid of 2
// to kRRMax columns that are not a level's tail (cid % 1024 == 1023).
constexpr int kRRMax = 16;

// Size of the cid run that holds column i when it is such a cluster (first
// column -> *first), else 0.
__device__ __forceinline__ int rr_cluster(const int32_t* __restrict__ cid, int k, int i, int* first) {
  const int id = cid[i];
  if ((id & 1023) == 1023) return 0;
  int a = i, b = i + 1;
  while (a > 0 && cid[a - 1] == id && i - a < kRRMax) --a;
  while (b < k && cid[b] == id && b - i <= kRRMax) ++b;
  const int sc = b - a;
  *first = a;
  return (sc >= 2 && sc <= kRRMax) ? sc : 0;
}

// Rayleigh-Ritz inside each small seed cluster: the eigenvectors Z of the
// cluster's block of S (symmetrised, FP64 cyclic Jacobi, one warp) are
// written to Zr[C, C] (cluster_rotate_kernel applies them).  The FP32 seed
// cannot order vectors whose eigenvalues are closer than its resolution; in
// FP64 they may well be distinct.
__global__ void __launch_bounds__(32) cluster_rr_kernel(const double* __restrict__ S, const int32_t* __restrict__ cid,
                                                        int k, double* __restrict__ Zr, const int32_t* act) {
  pdl_wait();  // first, on every path: completion stays ordered along the chain
  if (act && *act < 2) return;
  const int c = blockIdx.x, lane = threadIdx.x;
  int i0 = 0;
  const int sc = rr_cluster(cid, k, c, &i0);
  if (sc == 0 || i0 != c) return;  // one warp per cluster: its first column
  __shared__ double A[kRRMax][kRRMax + 1], Z[kRRMax][kRRMax + 1];
  __shared__ double cs[3];
  for (int e = lane; e < sc * sc; e += 32) {
    const int a = e / sc, b = e % sc;
    A[a][b] = 0.5 * (S[(int64_t)(i0 + a) * k + i0 + b] + S[(int64_t)(i0 + b) * k + i0 + a]);
    Z[a][b] = a == b ? 1.0 : 0.0;
  }
  __syncwarp();
  for (int sweep = 0; sweep < 12; ++sweep) {
    double off = 0.0, dia = 0.0;
    for (int e = lane; e < sc * sc; e += 32) {
      const int a = e / sc, b = e % sc;
      if (a != b) off += A[a][b] * A[a][b];
      else dia += A[a][b] * A[a][b];
    }
    off = warp_sum(off);
    dia = warp_sum(dia);
    if (!(off > 1e-30 * dia)) break;  // uniform
    for (int p = 0; p < sc - 1; ++p)
      for (int q = p + 1; q < sc; ++q) {
        if (lane == 0) {
          const double apq = A[p][q];
          double cc = 1.0, ss = 0.0, tt = 0.0;
          if (fabs(apq) > 1e-300) {
            const double th = (A[q][q] - A[p][p]) / (2.0 * apq);
            tt = (th >= 0.0 ? 1.0 : -1.0) / (fabs(th) + sqrt(th * th + 1.0));
            cc = 1.0 / sqrt(tt * tt + 1.0);
            ss = tt * cc;
          }
          cs[0] = cc;
          cs[1] = ss;
          cs[2] = tt;
        }
        __syncwarp();
        const double cc = cs[0], ss = cs[1], tt = cs[2];
        if (ss != 0.0) {
          const int r = lane;
          double arp = 0.0, arq = 0.0, zrp = 0.0, zrq = 0.0;
          if (r < sc) {
            arp = A[r][p];
            arq = A[r][q];
            zrp = Z[r][p];
            zrq = Z[r][q];
          }
          const double app = A[p][p], aqq = A[q][q], apq = A[p][q];
          __syncwarp();
          if (r < sc) {
            if (r != p && r != q) {
              const double np = cc * arp - ss * arq, nq = ss * arp + cc * arq;
              A[r][p] = np;
              A[p][r] = np;
              A[r][q] = nq;
              A[q][r] = nq;
            }
            Z[r][p] = cc * zrp - ss * zrq;
            Z[r][q] = ss * zrp + cc * zrq;
          }
          if (lane == 0) {
            A[p][p] = app - tt * apq;
            A[q][q] = aqq + tt * apq;
            A[p][q] = 0.0;
            A[q][p] = 0.0;
          }
        }
        __syncwarp();
      }
  }
  for (int e = lane; e < sc * sc; e += 32) {
    const int a = e / sc, b = e % sc;
    Zr[(int64_t)(i0 + a) * k + i0 + b] = Z[a][b];
  }
}

// Columns of each small seed cluster of X rotated in place by the cluster's
// Rayleigh-Ritz vectors: X[:, C] <- X[:, C] Zr[C, C], one CTA per row of X.
// It follows the first-order step X + X E, which leaves the cluster's span
// decoupled from the other columns; a rotation inside that span keeps it so.
// blockIdx.y selects the matrix: X, then (nullable) A1, A2.
__global__ void cluster_rotate_kernel(double* __restrict__ X, double* __restrict__ A1, double* __restrict__ A2,
                                      const int32_t* __restrict__ cid, const double* __restrict__ Zr, int k,
                                      const int32_t* act) {
  pdl_wait();  // first, on every path: completion stays ordered along the chain
  if (act && *act < 2) return;
  double* M = blockIdx.y == 0 ? X : (blockIdx.y == 1 ? A1 : A2);
  if (!M) return;
  const int r = blockIdx.x;
  for (int c = threadIdx.x; c < k; c += blockDim.x) {
    int i0 = 0;
    const int sc = rr_cluster(cid, k, c, &i0);
    if (sc == 0 || i0 != c) continue;
    double x[kRRMax], y[kRRMax];
    for (int a = 0; a < sc; ++a) x[a] = M[(int64_t)r * k + i0 + a];
    for (int b = 0; b < sc; ++b) {
      double t = 0.0;
      for (int a = 0; a < sc; ++a) t = fma(x[a], Zr[(int64_t)(i0 + a) * k + i0 + b], t);
      y[b] = t;
    }
    for (int b = 0; b < sc; ++b) M[(int64_t)r * k + i0 + b] = y[b];
  }
}

// Rows of each small cluster of A1 and A2 rotated in place: A[C, :] <-
// Zr[C, C]^T A[C, :], one CTA per column (with the column rotation above:
// A <- B^T A B for the block-diagonal B of the clusters' Rayleigh-Ritz vectors).
__global__ void cluster_rotate_rows_kernel(double* __restrict__ A1, double* __restrict__ A2,
                                           const int32_t* __restrict__ cid, const double* __restrict__ Zr, int k,
                                           const int32_t* act) {
  pdl_wait();  // first, on every path: completion stays ordered along the chain
  if (act && *act < 2) return;
  double* M = blockIdx.y == 0 ? A1 : A2;
  const int col = blockIdx.x;
  for (int c = threadIdx.x; c < k; c += blockDim.x) {
    int i0 = 0;
    const int sc = rr_cluster(cid, k, c, &i0);
    if (sc == 0 || i0 != c) continue;
    double x[kRRMax], y[kRRMax];
    for (int a = 0; a < sc; ++a) x[a] = M[(int64_t)(i0 + a) * k + col];
    for (int b = 0; b < sc; ++b) {
      double t = 0.0;
      for (int a = 0; a < sc; ++a) t = fma(Zr[(int64_t)(i0 + a) * k + i0 + b], x[a], t);
      y[b] = t;
    }
    for (int b = 0; b < sc; ++b) M[(int64_t)(i0 + b) * k + col] = y[b];
  }
}

// One refinement step's correction E, row i per block (R = I - Rm).  Pairs
// inside a level's unresolved tail, or inside a seed cluster of at most kRRMax
// columns, are only re-orthogonalised (r_ij / 2): the next level resolves the
// tail, and the Rayleigh-Ritz rotation (cluster_rr_kernel,
// cluster_rotate_kernel) the small cluster.  Any other pair -- also inside a
// larger seed cluster, where the gap must also exceed 1e-12 ||H||_F -- takes
// the first-order correction
// (s_ij + lambda_j r_ij) / (lambda_j - lambda_i) when that is a small
// rotation (|E_ij| <= 1/2) and the gap is above FP64 noise of H
// (64 eps ||H||_F, scal[1] = ||H||_F); otherwise it too is only
// re-orthogonalised.  The per-pair test replaces the method's global cluster
// threshold, which (evaluated with Frobenius norms) would leave close but
// well-coupled pairs unresolved; the iteration still converges quadratically
// for resolved pairs.  The Rayleigh quotients lambda are formed here from the
// diagonals of S and Rm (as rayleigh_kernel does), so the step needs no
// separate launch for them.
__global__ void refine_e_kernel(const double* __restrict__ Rm, const double* __restrict__ S,
                                const double* __restrict__ scal, const int32_t* __restrict__ cid, int k,
                                double* __restrict__ E, const int32_t* act) {
  pdl_wait();  // first, on every path: completion stays ordered along the chain
  if (act && *act < 2) return;
  const int i = blockIdx.x;
  const double noise = 64.0 * 0x1p-52 * scal[1];
  const double li = S[(int64_t)i * k + i] / Rm[(int64_t)i * k + i];
  const int ci = cid[i];
  int i0 = 0;
  // pairs held apart from the first-order step: a level's tail, a small cluster
  const bool held = (ci & 1023) == 1023 || rr_cluster(cid, k, i, &i0) != 0;
  // inside a larger cluster, a pair closer than this is degenerate in FP64
  const double degen = 1e-12 * scal[1];
  for (int j = threadIdx.x; j < k; j += blockDim.x) {
    const int64_t e = (int64_t)i * k + j;
    const double r = (i == j ? 1.0 : 0.0) - Rm[e];
    double v = 0.5 * r;
    const bool same = cid[j] == ci;
    if (i != j && !(held && same)) {
      const double lj = S[(int64_t)j * k + j] / Rm[(int64_t)j * k + j];
      const double gap = lj - li;
      const double num = S[e] + lj * r;
      if (fabs(gap) > (same ? degen : noise) && fabs(num) <= 0.5 * fabs(gap)) v = num / gap;
    }
    E[e] = v;
  }
}

// Sort eigenpairs by descending lambda (stable) and apply the rank rule; write
// sigma (device output), the column-permuted eigenvector matrix Ws and the
// k x k factor Tinv with V = F^T Ws Tinv.  With S = Ws^T H Ws, Tinv is the
// first-order inverse of the symmetric square root T of S:
//   T = D_s + Y,  D_s = diag(sqrt(S_rr)),  Y_ab = S_ab / (s_a + s_b)  (a != b),
//   Tinv = D_s^-1 - D_s^-1 Y D_s^-1,
// so V^T V = Tinv^T S Tinv = I up to O(|Y|^2) even where close eigenvalues
// leave W mixing a cluster (the denominators are sums, not gaps).  For an
// exactly diagonalising W this is the paper's D^-1.
__global__ void sort_rank_kernel(const double* __restrict__ lam, const double* __restrict__ S, int k, int64_t m,
                                 int64_t n, double* __restrict__ sigma, int32_t* rank, double* scal) {
  pdl_wait();  // first, on every path: completion stays ordered along the chain
  __shared__ double key[256];
  __shared__ int src[256];
  __shared__ double wmax[32];
  int32_t* src_g = reinterpret_cast<int32_t*>(scal + 8 + 2 * k);
  double* sd_g = scal + 8 + k;
  const int tid = threadIdx.x;
  // total order: NaN keys rank as -inf, ties by index, so the positions form a permutation
  double mx = 0.0;
  for (int i = tid; i < k; i += blockDim.x) {
    const double v = lam[i];
    key[i] = isnan(v) ? -INFINITY : v;
    mx = fmax(mx, key[i]);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if ((tid & 31) == 0) wmax[tid >> 5] = mx;
  __syncthreads();
  double lmax = 0.0;
  for (int w = 0; w < (int)(blockDim.x >> 5); ++w) lmax = fmax(lmax, wmax[w]);
  for (int i = tid; i < k; i += blockDim.x) {
    const double li = key[i];
    int pos = 0;
    for (int j = 0; j < k; ++j) {
      const double lj = key[j];
      pos += (lj > li) || (lj == li && j < i);
    }
    src[pos] = i;
  }
  __syncthreads();
  const double tol = (double)(m > n ? m : n) * 0x1p-52 * lmax;
  int kept = 0;
  for (int r = tid; r < k; r += blockDim.x) {
    const int i = src[r];
    const bool keep = lam[i] > tol && lmax > 0.0;  // false for NaN
    if (sigma) sigma[r] = keep ? sqrt(lam[i]) : 0.0;
    scal[8 + r] = keep ? sqrt(lam[i]) : 0.0;
    const double sii = S[(int64_t)i * k + i];
    sd_g[r] = (keep && sii > 0.0) ? sqrt(sii) : 0.0;
    src_g[r] = i;
    kept += keep;
  }
  __shared__ int wsum[32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) kept += __shfl_xor_sync(0xffffffffu, kept, o);
  if ((tid & 31) == 0) wsum[tid >> 5] = kept;
  __syncthreads();
  if (tid == 0) {
    int rk = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) rk += wsum[w];
    if (rank) *rank = rk;
    scal[0] = (double)rk;
  }
}

// Row a of Ws (column-permuted eigenvectors) and of Tinv, the first-order
// inverse of the symmetric square root T of S = Ws^T H Ws:
//   T = D_s + Y, D_s = diag(sqrt(S_rr)), Y_ab = S_ab / (s_a + s_b) (a != b),
//   Tinv = D_s^-1 - D_s^-1 Y D_s^-1.
// V = F^T Ws Tinv then has V^T V = Tinv^T S Tinv = I up to O(|Y|^2), also where
// close eigenvalues leave W mixing a cluster (the denominators are sums, not
// gaps).  For an exactly diagonalising W this is the paper's D^-1.
__global__ void ws_tinv_kernel(const double* __restrict__ W, const double* __restrict__ S,
                               const double* __restrict__ scal, int k, double* __restrict__ Ws,
                               double* __restrict__ Tinv, int* vcount) {
  pdl_wait();  // first, on every path: completion stays ordered along the chain
  const int a = blockIdx.x;
  // the arrival counters of vprod_kernel's column tiles start each call at zero
  if (vcount && a == 0 && threadIdx.x < (k + kVT - 1) / kVT) vcount[threadIdx.x] = 0;
  const int32_t* src = reinterpret_cast<const int32_t*>(scal + 8 + 2 * k);
  const double* sd = scal + 8 + k;
  const double sa = sd[a];
  for (int b = threadIdx.x; b < k; b += blockDim.x) {
    Ws[(int64_t)a * k + b] = W[(int64_t)a * k + src[b]];
    double t = 0.0;
    const double sb = sd[b];
    if (sa > 0.0 && sb > 0.0) {
      if (a == b) t = 1.0 / sa;
      else t = -S[(int64_t)src[a] * k + src[b]] / ((sa + sb) * sa * sb);
    }
    Tinv[(int64_t)a * k + b] = t;
  }
}

// FP32 V = F^T M (F k x n FP64, M = Ws Tinv k x k FP64) with the sign rule,
// in two launches.  vprod_kernel: one CTA per 64 x 64 tile of V; F^T and M
// staged whole over K = k in shared memory as FP32, 4 x 4 outputs per thread,
// products summed over 16-term slabs and the slab sums added to the running
// sum (the rounding of the previous SIMT product).  The tile is written
// unsigned, and each column's entry of largest magnitude over the tile (ties
// to the lowest row) goes to a partial; the last CTA of a column tile to
// arrive (a counter, zeroed by ws_tinv_kernel) reduces the partials of its
// columns in row order and writes each column's sign.  vsign_kernel negates
// the columns whose chosen entry is negative.
struct ColMax {
  float v;  // signed value of the largest-magnitude entry
  int i;    // its row
};

__global__ void __launch_bounds__(256) vprod_kernel(const double* __restrict__ F, int64_t n, int k,
                                                    const double* __restrict__ M, float* __restrict__ V,
                                                    ColMax* __restrict__ part, int* vcount, float* __restrict__ sgn) {
  pdl_wait();  // first, on every path: completion stays ordered along the chain
  extern __shared__ float vsm[];
  constexpr int LD = kVT + 4;
  float* As = vsm;            // [k][LD]: As[q][r] = F[q][r0 + r]
  float* Bs = vsm + k * LD;   // [k][LD]: Bs[q][c] = M[q][c0 + c]
  __shared__ ColMax red[16][kVT];
  __shared__ int last_s;
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const int64_t r0 = (int64_t)blockIdx.x * kVT;
  const int c0 = blockIdx.y * kVT;
  for (int e = tid; e < k * kVT; e += 256) {
    const int q = e / kVT, r = e % kVT;
    As[q * LD + r] = (r0 + r < n) ? (float)F[(int64_t)q * n + r0 + r] : 0.f;
    Bs[q * LD + r] = (c0 + r < k) ? (float)M[(int64_t)q * k + c0 + r] : 0.f;
  }
  __syncthreads();
  float acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = 0.f;
  for (int q0 = 0; q0 < k; q0 += 16) {
    float pt[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) pt[i][j] = 0.f;
    const int qe = min(k, q0 + 16);
    for (int q = q0; q < qe; ++q) {
      const float4 a = *reinterpret_cast<const float4*>(As + q * LD + ty * 4);
      const float4 b = *reinterpret_cast<const float4*>(Bs + q * LD + tx * 4);
      const float av[4] = {a.x, a.y, a.z, a.w}, bv[4] = {b.x, b.y, b.z, b.w};
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) pt[i][j] = fmaf(av[i], bv[j], pt[i][j]);
    }
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) acc[i][j] += pt[i][j];
  }
  // write the tile; per column the largest |v| of this thread's rows
  ColMax best[4];
#pragma unroll
  for (int j = 0; j < 4; ++j) best[j] = ColMax{0.f, -1};
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int64_t gr = r0 + ty * 4 + i;
    if (gr >= n) break;
    const int gc = c0 + tx * 4;
    if (gc + 4 <= k && (k & 3) == 0 && ((uintptr_t)V & 15) == 0) {
      *reinterpret_cast<float4*>(V + gr * k + gc) = make_float4(acc[i][0], acc[i][1], acc[i][2], acc[i][3]);
    } else {
#pragma unroll
      for (int j = 0; j < 4; ++j)
        if (gc + j < k) V[gr * k + gc + j] = acc[i][j];
    }
#pragma unroll
    for (int j = 0; j < 4; ++j)
      if (best[j].i < 0 || fabsf(acc[i][j]) > fabsf(best[j].v)) best[j] = ColMax{acc[i][j], (int)gr};
  }
#pragma unroll
  for (int j = 0; j < 4; ++j) red[ty][tx * 4 + j] = best[j];
  __syncthreads();
  if (tid < kVT) {
    ColMax b{0.f, -1};
    for (int y = 0; y < 16; ++y) {
      const ColMax o = red[y][tid];
      if (o.i >= 0 && (b.i < 0 || fabsf(o.v) > fabsf(b.v))) b = o;
    }
    if (c0 + tid < k) part[(int64_t)blockIdx.x * k + c0 + tid] = b;
  }
  __threadfence();
  __syncthreads();
  if (tid == 0) last_s = atomicAdd(&vcount[blockIdx.y], 1) == (int)gridDim.x - 1;
  __syncthreads();
  if (!last_s) return;
  __threadfence();
  if (tid < kVT && c0 + tid < k) {
    const int c = c0 + tid;
    ColMax b{0.f, -1};
    for (unsigned rt = 0; rt < gridDim.x; ++rt) {
      const ColMax* pp = part + (int64_t)rt * k + c;
      const ColMax o{__ldcg(&pp->v), __ldcg(&pp->i)};
      if (o.i >= 0 && (b.i < 0 || fabsf(o.v) > fabsf(b.v))) b = o;
    }
    sgn[c] = (b.v < 0.f) ? -1.f : 1.f;
  }
}

__global__ void __launch_bounds__(256) vsign_kernel(float* __restrict__ V, int64_t n, int k,
                                                    const float* __restrict__ sgn) {
  pdl_wait();  // first, on every path: completion stays ordered along the chain
  const int64_t total = n * k;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x)
    if (sgn[e % k] < 0.f) V[e] = -V[e];
}

// Sign rule and FP32 output: one block per column of Vd (n x k FP64).
template <typename VT>
__global__ void finalize_v_kernel(const double* __restrict__ Vd, int64_t n, int k, VT* __restrict__ V) {
  pdl_wait();  // first, on every path: completion stays ordered along the chain
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

// FP64 GEMM for the k x k step: C[z] = op(A) op(B) over the K range of split z,
// op(A)(r, q) = at ? A[q lda + r] : A[r lda + q], op(B)(q, c) = bt ? B[c ldb + q]
// : B[q ldb + c].  One CTA per TM x TN output tile (TM TN threads, one output
// each, four interleaved partial sums); K in slabs of KS staged whole in
// shared memory.  GB300 issues few FP64 FMAs per SM per clock, so the tiles
// are small enough to spread even a 128 x 128 product over all SMs.  sym:
// C is symmetric (op(B) = op(A)^T); only tiles with blockIdx.x <= blockIdx.y
// run and each also writes its mirror.  act (nullable): a seed level's block
// size on the device; below 2 the product is skipped and C = dflt when dflt is
// given (else C is left as it is).
struct DgemmArgs {
  int64_t M, N, K;
  const double* A;
  int64_t lda;
  int at;
  const double* B;
  int64_t ldb;
  int bt;
  double* C;
  int64_t ldc;
  int64_t c_split_stride, kchunk;
  int sym;
  const double* Cin;  // nullable: C = Cin + op(A) op(B)
  const int32_t* act;
  const double* dflt;
};

template <int TM, int TN, int KS>
__device__ __forceinline__ void dgemm_tile_body(const DgemmArgs& g, int z) {
  if (g.sym && blockIdx.x > blockIdx.y) return;
  if (g.act && *g.act < 2) {
    if (g.dflt && z == 0) {
      const int64_t gi = (int64_t)blockIdx.x * TM + threadIdx.x / TN, gj = (int64_t)blockIdx.y * TN + threadIdx.x % TN;
      if (gi < g.M && gj < g.N) g.C[gi * g.ldc + gj] = g.dflt[gi * g.ldc + gj];
    }
    return;
  }
  __shared__ double As[TM][KS + 1];
  __shared__ double Bs[TN][KS + 1];
  const int tid = threadIdx.x;
  const int r = tid / TN, c = tid % TN;
  const int64_t i0 = (int64_t)blockIdx.x * TM, j0 = (int64_t)blockIdx.y * TN;
  const int64_t kb = (int64_t)z * g.kchunk;
  const int64_t ke = min(g.K, kb + g.kchunk);
  double acc[4] = {0.0, 0.0, 0.0, 0.0};
  for (int64_t k0 = kb; k0 < ke; k0 += KS) {
    for (int e = tid; e < TM * KS; e += TM * TN) {
      int rr, q;
      if (g.at) { q = e / TM; rr = e % TM; } else { rr = e / KS; q = e % KS; }
      const int64_t gi = i0 + rr, gq = k0 + q;
      As[rr][q] = (gi < g.M && gq < ke) ? (g.at ? g.A[gq * g.lda + gi] : g.A[gi * g.lda + gq]) : 0.0;
    }
    for (int e = tid; e < TN * KS; e += TM * TN) {
      int cc, q;
      if (g.bt) { cc = e / KS; q = e % KS; } else { q = e / TN; cc = e % TN; }
      const int64_t gj = j0 + cc, gq = k0 + q;
      Bs[cc][q] = (gj < g.N && gq < ke) ? (g.bt ? g.B[gj * g.ldb + gq] : g.B[gq * g.ldb + gj]) : 0.0;
    }
    __syncthreads();
#pragma unroll 4
    for (int q = 0; q < KS; q += 4) {
#pragma unroll
      for (int u = 0; u < 4; ++u) acc[u] = fma(As[r][q + u], Bs[c][q + u], acc[u]);
    }
    __syncthreads();
  }
  double v = (acc[0] + acc[1]) + (acc[2] + acc[3]);
  double* Cs = g.C + (int64_t)z * g.c_split_stride;
  const int64_t gi = i0 + r, gj = j0 + c;
  if (gi < g.M && gj < g.N) {
    if (g.Cin) v += g.Cin[gi * g.ldc + gj];
    Cs[gi * g.ldc + gj] = v;
    if (g.sym && blockIdx.x != blockIdx.y) Cs[gj * g.ldc + gi] = v;
  }
}

// blockIdx.z: the K split.
template <int TM, int TN, int KS>
__global__ void __launch_bounds__(TM* TN) dgemm_tile_kernel(const DgemmArgs g) {
  pdl_wait();  // first, on every path: completion stays ordered along the chain
  dgemm_tile_body<TM, TN, KS>(g, blockIdx.z);
}

// Two independent products in one launch (blockIdx.z selects), K unsplit.
template <int TM, int TN, int KS>
__global__ void __launch_bounds__(TM* TN) dgemm_pair_kernel(const DgemmArgs g0, const DgemmArgs g1) {
  pdl_wait();  // first, on every path: completion stays ordered along the chain
  dgemm_tile_body<TM, TN, KS>(blockIdx.z == 0 ? g0 : g1, 0);
}

static DgemmArgs dargs(int64_t M, int64_t N, int64_t K, const double* A, int64_t lda, bool at, const double* B,
                       int64_t ldb, bool bt, double* C, int64_t ldc, const double* Cin = nullptr,
                       const int32_t* act = nullptr, const double* dflt = nullptr) {
  DgemmArgs g{};
  g.M = M;
  g.N = N;
  g.K = K;
  g.A = A;
  g.lda = lda;
  g.at = at ? 1 : 0;
  g.B = B;
  g.ldb = ldb;
  g.bt = bt ? 1 : 0;
  g.C = C;
  g.ldc = ldc;
  g.c_split_stride = 0;
  g.kchunk = K;
  g.sym = 0;
  g.Cin = Cin;
  g.act = act;
  g.dflt = dflt;
  return g;
}

// Both products are M x N.
static void dgemm2(Launcher& L, const DgemmArgs& g0, const DgemmArgs& g1) {
  dim3 grid((unsigned)((g0.M + 7) / 8), (unsigned)((g0.N + 7) / 8), 2);
  launch_pdl(L, dgemm_pair_kernel<8, 8, 64>, dim3(grid), dim3(64), 0, g0, g1);
  L.count(1);
}

static void dgemm(Launcher& L, int64_t M, int64_t N, int64_t K, const double* A, int64_t lda, bool at, const double* B,
                  int64_t ldb, bool bt, double* C, int64_t ldc, const double* Cin = nullptr,
                  const int32_t* act = nullptr, const double* dflt = nullptr, bool sym = false) {
  dim3 grid((unsigned)((M + 7) / 8), (unsigned)((N + 7) / 8), 1);
  DgemmArgs g = dargs(M, N, K, A, lda, at, B, ldb, bt, C, ldc, Cin, act, dflt);
  g.sym = sym ? 1 : 0;
  launch_pdl(L, dgemm_tile_kernel<8, 8, 64>, dim3(grid), dim3(64), 0, g);
  L.count(1);
}

static DgemmArgs sym_args(DgemmArgs g) {
  g.sym = 1;
  return g;
}

void launch_decompose(Launcher& L, SmallWs& w, const double* F, int k, int64_t n, int64_t m, bool v_f64, void* V,
                      double* sigma, int32_t* rank, int* status) {
  const int64_t kk = (int64_t)k * k;
  // H = F F^T.  FP32-class results (FP32 V): on the tensor cores from exact
  // digit planes of F (ozaki.cu).  FP64 V: FP64 SIMT products split over n,
  // upper tiles mirrored, reduced in fixed order.
  if (!v_f64) {
    launch_oz_gram(L, F, k, n, w.oz, w.H, status);
  } else {
    const int64_t kchunk = ((n + w.h_splits - 1) / w.h_splits + 63) / 64 * 64;
    dim3 grid((unsigned)((k + 15) / 16), (unsigned)((k + 15) / 16), (unsigned)w.h_splits);
    DgemmArgs g = dargs(k, k, n, F, n, false, F, n, true, w.Hpart, k);
    g.c_split_stride = kk;
    g.kchunk = kchunk;
    g.sym = 1;
    launch_pdl(L, dgemm_tile_kernel<16, 16, 64>, dim3(grid), dim3(256), 0, g);
    L.count(1);
    launch_reduce_splits(L, w.Hpart, w.h_splits, kk, kk, w.H);
  }
  // Graded eigensolve: level 0 seeds H; each later level seeds the tail block
  // of S = X^T H X left unresolved by the level before, and rotates those
  // columns of X; every level ends with the FP64 refinement.
  double* X = w.Xa;
  double* Xn = w.Xb;
  for (int level = 0; level < kSeedLevels; ++level) {
    const int32_t* act = level == 0 ? nullptr : w.lvl + level;
    if (level == 0) {
      launch_seed_level(L, w.H, k, 0, w.lvl, w.h32, w.w32, w.q32, w.p32, w.tri, X, w.lam, w.scal, w.sweeps,
                        w.cid);
    } else {
      launch_seed_level(L, w.S, k, level, w.lvl, w.h32, w.w32, w.q32, w.p32, w.tri, w.E, w.lam, w.scal, w.sweeps,
                        w.cid);
      dgemm(L, k, k, k, X, k, false, w.E, k, false, Xn, k, nullptr, act, X);  // X blockdiag(W, I)
      double* t = X;
      X = Xn;
      Xn = t;
    }
    // FP64 refinement
    for (int it = 0; it <= kRefineIters; ++it) {
      dgemm2(L, sym_args(dargs(k, k, k, X, k, true, X, k, false, w.Rm, k, nullptr, act)),  // X^T X
             dargs(k, k, k, w.H, k, false, X, k, false, w.T, k, nullptr, act));            // H X
      // X^T (H X): symmetric up to rounding; the upper triangle is mirrored
      dgemm(L, k, k, k, X, k, true, w.T, k, false, w.S, k, nullptr, act, nullptr, true);
      if (it == kRefineIters) {
        // last pass: a final Rayleigh-Ritz rotation of the small clusters,
        // applied to X, S and X^T X alike (B^T S B), then lambda
        launch_pdl(L, cluster_rr_kernel, dim3(k), dim3(32), 0, w.S, w.cid, k, w.T, act);
        launch_pdl(L, cluster_rotate_kernel, dim3(k, 3), dim3(64), 0, X, w.S, w.Rm, w.cid, w.T, k, act);
        launch_pdl(L, cluster_rotate_rows_kernel, dim3(k, 2), dim3(64), 0, w.S, w.Rm, w.cid, w.T, k, act);
        launch_pdl(L, rayleigh_kernel, dim3(1), dim3(256), 0, w.Rm, w.S, k, w.lam, act);
        L.count(4);
        break;
      }
      // T (H X) is free once S is formed: it holds the clusters' Rayleigh-Ritz vectors
      launch_pdl(L, cluster_rr_kernel, dim3(k), dim3(32), 0, w.S, w.cid, k, w.T, act);
      launch_pdl(L, refine_e_kernel, dim3(k), dim3(128), 0, w.Rm, w.S, w.scal, w.cid, k, w.E, act);
      L.count(2);
      dgemm(L, k, k, k, X, k, false, w.E, k, false, Xn, k, X, act, X);  // X + X E
      launch_pdl(L, cluster_rotate_kernel, dim3(k, 1), dim3(64), 0, Xn, nullptr, nullptr, w.cid, w.T, k, act);
      L.count(1);
      double* t = X;
      X = Xn;
      Xn = t;
    }
  }
  // order, rank rule, Ws and Tinv (S of the final X is in w.S)
  launch_pdl(L, sort_rank_kernel, dim3(1), dim3(256), 0, w.lam, w.S, k, m, n, sigma, rank, w.scal);
  // FP32 V: the fused product and sign rule (vprod_kernel, vsign_kernel)
  const int nct = (k + kVT - 1) / kVT;
  const int64_t nrt = (n + kVT - 1) / kVT;
  ColMax* vpart = (ColMax*)w.vaux;
  float* vsgn = (float*)((char*)w.vaux + ((nrt * k * 8 + 255) / 256) * 256);
  int* vcount = (int*)((char*)vsgn + (((size_t)k * 4 + 255) / 256) * 256);
  launch_pdl(L, ws_tinv_kernel, dim3(k), dim3(128), 0, X, w.S, w.scal, k, w.T, w.E, v_f64 ? nullptr : vcount);
  L.count(2);
  dgemm(L, k, k, k, w.T, k, false, w.E, k, false, w.Rm, k);  // Ws Tinv
  // V = F^T (Ws Tinv)  (n x k): FP64 for an FP64 V; for an FP32 V (the result
  // type of FP32 / BF16 / E4M3 X) an FP32 product of the FP64 factors rounded
  // to FP32, summed over K in 16-term slabs (relative error ~1e-7 of an
  // FP32-rounded result); the factorisation itself stays FP64
  if (v_f64) {
    launch_gemm_simt(L, n, k, k, F, LSPCA_F64, n, true, w.Rm, LSPCA_F64, k, false, w.Vd, true, k, 0, 1, true, true);
    launch_pdl(L, finalize_v_kernel<double>, dim3(k), dim3(256), 0, w.Vd, n, k, (double*)V);
    L.count(1);
  } else {
    const size_t smem = (size_t)2 * k * (kVT + 4) * sizeof(float);
    cudaFuncSetAttribute(vprod_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    launch_pdl(L, vprod_kernel, dim3((unsigned)nrt, (unsigned)nct), dim3(256), smem, F, n, k, (const double*)w.Rm,
               (float*)V, vpart, vcount, vsgn);
    int blocks = (int)((n * k + 255) / 256);
    if (blocks > 4 * L.num_sms) blocks = 4 * L.num_sms;
    if (blocks < 1) blocks = 1;
    launch_pdl(L, vsign_kernel, dim3(blocks), dim3(256), 0, (float*)V, n, k, (const float*)vsgn);
    L.count(2);
  }
}

}  // namespace lspca
