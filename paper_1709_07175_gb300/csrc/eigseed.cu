// FP32 seed of the symmetric eigensolve of the k x k step.
//
// The FP64 refinement that follows (small.cu) needs eigenvectors accurate to
// well under a radian per pair; a standard dense symmetric route gives them in
// O(k^3) flops with O(k) synchronisations:
//   1. Householder tridiagonalisation  H = Q T Q^T;
//   2. eigenvalues of T by multisection on Sturm counts, to the resolution of
//      30 halvings of the Gershgorin interval;
//   3. eigenvectors of T by two steps of inverse iteration with an LDL^T solve
//      of T - lambda I; eigenvalues closer than 1e-5 ||T|| form a cluster whose
//      vectors are computed in order by one thread and Gram-Schmidt
//      orthogonalised against (up to 32 of) the cluster's earlier vectors, as
//      LAPACK's stein does (which uses 1e-3 ||T||: pairs between the two
//      thresholds come out non-orthogonal by at most ~1e-2 here, well inside
//      what the FP64 refinement corrects);
//   4. back-transformation W = Q Z.
// H is scaled by 1 / max|H_ii| first.
//
// k <= 128 runs as four launches (seed_*_kernel, below): the
// tridiagonalisation in registers on one CTA, the multisection with one warp
// per eigenvalue and the back-transformation with one warp per column on many
// SMs, the inverse iteration on one CTA.  k > 128 runs in one CTA
// (eig_seed_kernel) over a global scratch matrix: thread t maps to (group
// t / 256, column t % 256), so consecutive lanes touch consecutive addresses
// and every step needs at most four block barriers.
#include "common.cuh"
#include "kernels.h"

namespace lspca {

constexpr int kSeedThreads = 512;

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

// Register-resident form of step 1 for k <= 128: thread t owns the entries
// (r, c) with c = t mod 128 and r = t / 128 + 4 i, i = 0..31, of the matrix
// being reduced.  Vectors indexed by row are also kept "permuted",
// x[(r mod 4) * 32 + r / 4], so that a thread reads the 32 entries of its
// rows with eight 16-byte broadcast loads.
// Vectors are zero outside the active range, which makes every update a plain
// multiply-add over all 32 rows (no predicates).
__device__ __forceinline__ int perm_idx(int r) { return (r & 3) * 32 + (r >> 2); }

// Step 1: tridiagonalisation.  A (k x k, row-major, already scaled) is read
// from `Asrc`; the reflectors are left in Vh (row j: permuted v_j) and d, e,
// beta in dv, ev, betav.  Four barriers per reflector.
__device__ void tridiag_regs(const float* Asrc, int k, float* Vh, float* dv, float* ev, float* betav, float* rowbuf,
                             float* vfl, float* wl, float* vperm, float* wperm, float* gpart) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int tr = tid & 127, tg = tid >> 7;
  float a[32];
#pragma unroll
  for (int i = 0; i < 32; ++i) {
    const int r = tg + 4 * i;
    a[i] = (r < k && tr < k) ? Asrc[r * k + tr] : 0.f;
  }
  if (tg == 0) rowbuf[tr] = a[0];  // row 0
  __syncthreads();
  for (int j = 0; j + 2 < k; ++j) {
    // a. warp 0: reflector of row j (x = A[j][j+1..k-1])
    if (warp == 0) {
      float sq = 0.f;
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int r = lane + 32 * q;
        const float x = (r >= j + 2 && r < k) ? rowbuf[r] : 0.f;
        sq = fmaf(x, x, sq);
      }
      sq = warp_sumf(sq);
      const float x0 = rowbuf[j + 1];
      const float nrm = sqrtf(x0 * x0 + sq);
      float alpha = 0.f, beta = 0.f, v0 = x0;
      if (nrm > 0.f) {
        alpha = x0 >= 0.f ? -nrm : nrm;
        v0 = x0 - alpha;
        const float vv = v0 * v0 + sq;
        beta = vv > 0.f ? 2.f / vv : 0.f;
      }
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int r = lane + 32 * q;
        const float v = r == j + 1 ? v0 : ((r > j + 1 && r < k) ? rowbuf[r] : 0.f);
        vfl[r] = v;
        vperm[perm_idx(r)] = v;
        Vh[j * 128 + perm_idx(r)] = v;
      }
      if (lane == 0) {
        dv[j] = rowbuf[j];
        ev[j] = (nrm > 0.f) ? alpha : x0;
        betav[j] = beta;
      }
    }
    __syncthreads();
    const float beta = betav[j];
    // b. partial p_c = sum over the thread's rows of A[r][c] v_r
    {
      const float4* vp = reinterpret_cast<const float4*>(vperm + tg * 32);
      float s0 = 0.f, s1 = 0.f;
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        const float4 v = vp[q];
        s0 = fmaf(a[4 * q], v.x, s0);
        s1 = fmaf(a[4 * q + 1], v.y, s1);
        s0 = fmaf(a[4 * q + 2], v.z, s0);
        s1 = fmaf(a[4 * q + 3], v.w, s1);
      }
      gpart[tg * 128 + tr] = s0 + s1;
    }
    __syncthreads();
    // c. warp 0: p = beta A' v, K = beta p.v / 2, w = p - K v (zero outside rows j+1..k-1)
    if (warp == 0) {
      float pr[4], pv = 0.f;
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int r = lane + 32 * q;
        const bool act = r > j && r < k;
        const float p = act ? beta * (gpart[r] + gpart[128 + r] + gpart[256 + r] + gpart[384 + r]) : 0.f;
        pr[q] = p;
        pv = fmaf(p, vfl[r], pv);
      }
      pv = warp_sumf(pv);
      const float K = 0.5f * beta * pv;
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int r = lane + 32 * q;
        const float w = (r > j && r < k) ? pr[q] - K * vfl[r] : 0.f;
        wl[r] = w;
        wperm[perm_idx(r)] = w;
      }
    }
    __syncthreads();
    // d. A -= v w^T + w v^T; the owners of row j + 1 publish it for the next step
    {
      const float vc = vfl[tr], wc = wl[tr];
      const float4* vp = reinterpret_cast<const float4*>(vperm + tg * 32);
      const float4* wp = reinterpret_cast<const float4*>(wperm + tg * 32);
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        const float4 v = vp[q], w = wp[q];
        a[4 * q] -= v.x * wc + w.x * vc;
        a[4 * q + 1] -= v.y * wc + w.y * vc;
        a[4 * q + 2] -= v.z * wc + w.z * vc;
        a[4 * q + 3] -= v.w * wc + w.w * vc;
      }
#pragma unroll
      for (int i = 0; i < 32; ++i)
        if (tg + 4 * i == j + 1) rowbuf[tr] = a[i];
    }
    __syncthreads();
  }
  // the last 2 x 2 block (rows k-2, k-1), or the whole matrix when k < 3
#pragma unroll
  for (int i = 0; i < 32; ++i) {
    const int r = tg + 4 * i;
    if (r == k - 2 && tr < k) gpart[tr] = a[i];
    if (r == k - 1 && tr < k) gpart[128 + tr] = a[i];
  }
  __syncthreads();
  if (tid == 0) {
    if (k >= 2) {
      dv[k - 2] = gpart[k - 2];
      ev[k - 2] = gpart[128 + k - 2];
      betav[k - 2] = 0.f;
    }
    dv[k - 1] = gpart[128 + k - 1];
    betav[k - 1] = 0.f;
  }
  __syncthreads();
}

__global__ void __launch_bounds__(kSeedThreads, 1) eig_seed_kernel(const double* __restrict__ H, int k, float* gA,
                                                                float* gZ, float* gQ, double* __restrict__ Xout,
                                                                double* __restrict__ lam_out, double* scal,
                                                                int32_t* nclusters) {
  __shared__ float dv[256], ev[256], e2v[256], betav[256], wl[256], pv_s[256], lamv[256], vv_s[256];
  __shared__ float gpart[kSeedThreads];
  __shared__ float coef[4];
  __shared__ int clstart[257];
  float* A = gA;   // k x k row-major: scaled H, then the reflectors
  float* Z = gZ;   // k x k, column j = eigenvector j
  float* Qs = gQ;  // inverse-iteration scratch, one row per cluster
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = kSeedThreads / 32;

  // scale and load; ||H||_F for the refinement's noise floor
  __shared__ double hmax_s;
  __shared__ double hmx[kSeedThreads / 32];
  {
    double mx = 0.0;
    for (int i = tid; i < k; i += kSeedThreads) mx = fmax(mx, fabs(H[(int64_t)i * k + i]));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if (lane == 0) hmx[warp] = mx;
    __syncthreads();
    if (tid == 0) {
      double m2 = 0.0;
      for (int i = 0; i < nw; ++i) m2 = fmax(m2, hmx[i]);
      hmax_s = m2 > 0.0 ? m2 : 1.0;
    }
  }
  __syncthreads();
  const double sc = 1.0 / hmax_s;
  double hf = 0.0;
#pragma unroll 8
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

  // ---- 1. tridiagonalisation over the global scratch matrix
  const int kp = 256;                // padded width: thread t = (t / kp, t % kp)
  const int GR = kSeedThreads / kp;  // 2 groups
  const int tr = tid % kp, tg = tid / kp;
// Step j reflects the trailing block
  // A' = A[j+1:, j+1:] with H = I - beta v v^T built from row j (equal to
  // column j: the trailing block is kept whole and symmetric).  Four barriers
  // per step:
  //   a. warp 0: norm of row j right of the diagonal, alpha, beta, v (stored
  //      back into row j for the back-transformation and into vv_s);
  //   b. p = A' v: thread (g, r) sums a quarter (k <= 128) or half of the
  //      terms of p_r, reading A'[l][r] = A'[r][l] along rows (consecutive
  //      lanes, consecutive addresses);
  //   c. warp 0: p = beta sum of the partials, K = beta p.v / 2, w = p - K v;
  //   d. A' -= v w^T + w v^T, thread (g, c) over rows r = g mod GR.
  for (int j = 0; j + 2 < k; ++j) {
    const int n1 = k - j - 1;
    float* rowj = A + j * k + (j + 1);  // row j right of the diagonal (length n1)
    if (warp == 0) {
      float sq = 0.f;
      for (int r = 1 + lane; r < n1; r += 32) sq = fmaf(rowj[r], rowj[r], sq);
      sq = warp_sumf(sq);
      const float x0 = rowj[0];
      const float nrm = sqrtf(x0 * x0 + sq);
      float alpha = 0.f, beta = 0.f, v0 = x0;
      if (nrm > 0.f) {
        alpha = x0 >= 0.f ? -nrm : nrm;
        v0 = x0 - alpha;
        const float vv = v0 * v0 + sq;
        beta = vv > 0.f ? 2.f / vv : 0.f;
      }
      for (int r = lane; r < n1; r += 32) vv_s[r] = r == 0 ? v0 : rowj[r];
      __syncwarp();
      if (lane == 0) {
        dv[j] = A[j * k + j];
        ev[j] = (nrm > 0.f) ? alpha : x0;
        betav[j] = beta;
        rowj[0] = v0;
      }
    }
    __syncthreads();
    const float beta = betav[j];
    if (beta == 0.f) continue;  // uniform: the block is already reduced here
    const float* Ap = A + (j + 1) * k + (j + 1);
    {
      const int chunk = (n1 + GR - 1) / GR;
      const int l0 = tg * chunk, l1 = min(n1, l0 + chunk);
      float a0 = 0.f, a1 = 0.f;
      if (tr < n1) {
        int l = l0;
        for (; l + 1 < l1; l += 2) {
          a0 = fmaf(Ap[l * k + tr], vv_s[l], a0);
          a1 = fmaf(Ap[(l + 1) * k + tr], vv_s[l + 1], a1);
        }
        if (l < l1) a0 = fmaf(Ap[l * k + tr], vv_s[l], a0);
      }
      gpart[tg * kp + tr] = a0 + a1;
    }
    __syncthreads();
    if (warp == 0) {
      float pv = 0.f;
      for (int r = lane; r < n1; r += 32) {
        float s = 0.f;
        for (int g = 0; g < GR; ++g) s += gpart[g * kp + r];
        s *= beta;
        pv_s[r] = s;
        pv = fmaf(s, vv_s[r], pv);
      }
      pv = warp_sumf(pv);
      const float K = 0.5f * beta * pv;
      for (int r = lane; r < n1; r += 32) wl[r] = pv_s[r] - K * vv_s[r];
    }
    __syncthreads();
    if (tr < n1) {
      const float vc = vv_s[tr], wc = wl[tr];
      for (int r = tg; r < n1; r += GR) {
        float* a = A + (j + 1 + r) * k + (j + 1) + tr;
        *a -= vv_s[r] * wc + wl[r] * vc;
      }
    }
    __syncthreads();
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

  // ---- 2. eigenvalues by multisection: GR threads (lanes of one warp) per
  // eigenvalue evaluate Sturm counts at GR interior points of the bracket,
  // which shrinks by GR + 1 per round ((GR + 1)^rounds >= 2^30, the
  // resolution of 30 halvings of the Gershgorin interval).
  {
    const int idx = tid / GR, q = tid % GR;
    const int rounds = GR == 4 ? 13 : 19;
    const float den = (float)(GR + 1);
    float lo = coef[0], hi = coef[1];
#pragma unroll 1
    for (int it = 0; it < rounds; ++it) {
      const float x = lo + (hi - lo) * (float)(q + 1) / den;
      const bool above = idx < k && sturm_count(dv, e2v, k, x, pivmin) > idx;
      const unsigned ball = __ballot_sync(0xffffffffu, above);
      const unsigned grp = (ball >> ((lane / GR) * GR)) & ((1u << GR) - 1u);
      const int first = grp ? __ffs((int)grp) - 1 : GR;  // first point with count > idx
      const float nlo = first == 0 ? lo : lo + (hi - lo) * (float)first / den;
      const float nhi = first == GR ? hi : lo + (hi - lo) * (float)(first + 1) / den;
      lo = nlo;
      hi = nhi;
    }
    if (q == 0 && idx < k) lamv[idx] = 0.5f * (lo + hi);
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

  // ---- 4. back-transformation Z <- H_0 H_1 ... H_{k-3} Z, last reflector
  // first; v_j is row j of A right of the diagonal.  Thread (g, c), two
  // barriers per reflector:
  //   1. partial of w_c = v^T Z[j+1:, c] over the rows r = g mod GR;
  //   2. w_c = beta (sum of the GR partials of column c), then
  //      Z[j+1+r][c] -= v_r w_c over the same rows.
for (int j = k - 3; j >= 0; --j) {
    const float beta = betav[j];
    if (beta == 0.f) continue;
    const int n1 = k - j - 1;
    const float* v = A + j * k + (j + 1);
    float acc = 0.f;
    if (tr < k)
      for (int r = tg; r < n1; r += GR) acc = fmaf(v[r], Z[(j + 1 + r) * k + tr], acc);
    gpart[tg * kp + tr] = acc;
    __syncthreads();
    if (tr < k) {
      float wc = 0.f;
      for (int g = 0; g < GR; ++g) wc += gpart[g * kp + tr];
      wc *= beta;
      for (int r = tg; r < n1; r += GR) Z[(j + 1 + r) * k + tr] -= v[r] * wc;
    }
    __syncthreads();
  }
  for (int e = tid; e < k * k; e += kSeedThreads) Xout[e] = (double)Z[e];
  for (int i = tid; i < k; i += kSeedThreads) lam_out[i] = (double)lamv[i] * hmax_s;
}


// ---------------------------------------------------------------------------
// The same seed for k <= 128 in four launches, so that the steps that are
// independent across eigenvalues or columns run on many SMs instead of one:
//   seed_tri_kernel   (one CTA)        scale, load, steps 1 and the Gershgorin
//                                      interval; reflectors and T to global;
//   seed_bisect_kernel (k / 4 CTAs)    step 2, one warp per eigenvalue, 32
//                                      interior points per round (6 rounds,
//                                      33^6 >= 2^30: the resolution of 30
//                                      halvings);
//   seed_vec_kernel   (one CTA)        step 3, as in eig_seed_kernel;
//   seed_back_kernel  (k / 8 CTAs)     step 4, one warp per column of Z: the
//                                      reflectors applied one at a time with a
//                                      warp reduction each, no block barrier.
// Scratch `tri` (floats): d [0, k), e [k, 2k), e^2 [2k, 3k), beta [3k, 4k),
// eigenvalues of T [4k, 5k), then gl, gu, ||T||, pivmin, 1 / scale (as two
// floats: the FP64 max |H_ii| split hi + lo).  gA: reflector j in row j
// (k x k, zero outside rows j+1 .. k-1); gZ: eigenvectors of T (k x k, column
// i = vector i).

__global__ void __launch_bounds__(kSeedThreads, 1) seed_tri_kernel(const double* __restrict__ H, int k, float* gV,
                                                                float* tri, double* scal) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ float dv[256], ev[256], betav[256], wl[256];
  __shared__ float gpart[kSeedThreads];
  __shared__ __align__(16) float vperm[128], wperm[128];
  __shared__ float rowbuf[128], vfl[128];
  __shared__ double hmax_s;
  __shared__ double hmx[kSeedThreads / 32];
  __shared__ double redd[32];
  float* A = reinterpret_cast<float*>(smem_raw);  // 128 x k: scaled H, then the reflectors (permuted rows)
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = kSeedThreads / 32;
  {
    double mx = 0.0;
    for (int i = tid; i < k; i += kSeedThreads) mx = fmax(mx, fabs(H[(int64_t)i * k + i]));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if (lane == 0) hmx[warp] = mx;
    __syncthreads();
    if (tid == 0) {
      double m2 = 0.0;
      for (int i = 0; i < nw; ++i) m2 = fmax(m2, hmx[i]);
      hmax_s = m2 > 0.0 ? m2 : 1.0;
    }
  }
  __syncthreads();
  const double sc = 1.0 / hmax_s;
  double hf = 0.0;
#pragma unroll 8
  for (int e = tid; e < k * k; e += kSeedThreads) {
    const double h = H[e];
    hf += h * h;
    A[e] = (float)(h * sc);
  }
  hf = warp_sum(hf);
  if (lane == 0) redd[warp] = hf;
  __syncthreads();
  if (tid == 0) {
    double sum = 0.0;
    for (int i = 0; i < nw; ++i) sum += redd[i];
    scal[1] = sqrt(sum);
  }
  __syncthreads();
  tridiag_regs(A, k, A, dv, ev, betav, rowbuf, vfl, wl, vperm, wperm, gpart);
  // reflectors to global in natural order, T and its Gershgorin interval
  for (int e = tid; e < k * k; e += kSeedThreads) {
    const int j = e / k, r = e % k;
    gV[e] = A[j * 128 + perm_idx(r)];
  }
  for (int i = tid; i < k; i += kSeedThreads) {
    tri[i] = dv[i];
    tri[k + i] = ev[i];
    tri[2 * k + i] = (i + 1 < k) ? ev[i] * ev[i] : 0.f;
    tri[3 * k + i] = betav[i];
  }
  if (tid == 0) {
    float gl = 1e30f, gu = -1e30f, tn = 0.f;
    for (int i = 0; i < k; ++i) {
      const float off = (i > 0 ? fabsf(ev[i - 1]) : 0.f) + (i + 1 < k ? fabsf(ev[i]) : 0.f);
      gl = fminf(gl, dv[i] - off);
      gu = fmaxf(gu, dv[i] + off);
      tn = fmaxf(tn, fabsf(dv[i]) + off);
    }
    const float pad = 2.f * 1.2e-7f * tn + 1e-30f;
    float* c = tri + 5 * k;
    c[0] = gl - pad;
    c[1] = gu + pad;
    c[2] = tn;
    c[3] = fmaxf(1e-30f, 1.2e-7f * 1e-6f * tn);  // pivmin
    const float hi = (float)hmax_s;
    c[4] = hi;
    c[5] = (float)(hmax_s - (double)hi);
  }
}

// One warp per eigenvalue idx (ascending): Sturm counts at 32 interior points
// of the bracket per round.
__global__ void __launch_bounds__(128) seed_bisect_kernel(int k, float* tri) {
  __shared__ float d[128], e2[128];
  for (int i = threadIdx.x; i < k; i += blockDim.x) {
    d[i] = tri[i];
    e2[i] = tri[2 * k + i];
  }
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const int idx = blockIdx.x * 4 + (threadIdx.x >> 5);
  if (idx >= k) return;
  const float* c = tri + 5 * k;
  const float pivmin = c[3];
  float lo = c[0], hi = c[1];
#pragma unroll 1
  for (int it = 0; it < 6; ++it) {
    const float x = lo + (hi - lo) * (float)(lane + 1) / 33.f;
    const bool above = sturm_count(d, e2, k, x, pivmin) > idx;
    const unsigned ball = __ballot_sync(0xffffffffu, above);
    const int first = ball ? __ffs((int)ball) - 1 : 32;  // first point with count > idx
    const float nlo = first == 0 ? lo : lo + (hi - lo) * (float)first / 33.f;
    const float nhi = first == 32 ? hi : lo + (hi - lo) * (float)(first + 1) / 33.f;
    lo = nlo;
    hi = nhi;
  }
  if (lane == 0) tri[4 * k + idx] = 0.5f * (lo + hi);
}

// Step 3 of eig_seed_kernel (clusters, inverse iteration, Gram-Schmidt inside
// clusters) for k <= 128: Z and the per-cluster scratch in shared memory.
__global__ void __launch_bounds__(128, 1) seed_vec_kernel(int k, const float* __restrict__ tri, float* gZ,
                                                        int32_t* nclusters) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ float dv[128], ev[128], lamv[128];
  __shared__ int clstart[130];
  float* Z = reinterpret_cast<float*>(smem_raw);  // k x k, column i = eigenvector i
  float* Qs = Z + k * k;                          // one row per cluster
  const int tid = threadIdx.x;
  for (int i = tid; i < k; i += blockDim.x) {
    dv[i] = tri[i];
    ev[i] = tri[k + i];
    lamv[i] = tri[4 * k + i];
  }
  __syncthreads();
  const float tnorm = tri[5 * k + 2], pivmin = tri[5 * k + 3];
  if (tid == 0) {
    int nc = 0;
    for (int i = 0; i < k; ++i)
      if (i == 0 || lamv[i] - lamv[i - 1] > 1e-5f * tnorm) clstart[nc++] = i;
    clstart[nc] = k;
    clstart[129] = nc;
    *nclusters = nc;
  }
  __syncthreads();
  const int ncl = clstart[129];
  for (int cl = tid; cl < ncl; cl += blockDim.x) {
    const int i0 = clstart[cl], i1 = clstart[cl + 1];
    float* q = Qs + cl;
    for (int i = i0; i < i1; ++i) {
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
  for (int e = tid; e < k * k; e += blockDim.x) gZ[e] = Z[e];
}

// Step 4, one warp per column c of Z: z <- H_0 H_1 ... H_{k-3} z, lane l
// holding rows l, l + 32, l + 64, l + 96; eigenvalues scaled back into lam.
__global__ void __launch_bounds__(256) seed_back_kernel(int k, const float* __restrict__ gV,
                                                      const float* __restrict__ gZ, const float* __restrict__ tri,
                                                      double* __restrict__ Xout, double* __restrict__ lam_out) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float* Vs = reinterpret_cast<float*>(smem_raw);  // k x k reflectors
  __shared__ float beta[128];
  for (int e = threadIdx.x; e < k * k; e += blockDim.x) Vs[e] = gV[e];
  for (int i = threadIdx.x; i < k; i += blockDim.x) beta[i] = tri[3 * k + i];
  __syncthreads();
  const double hmax = (double)tri[5 * k + 4] + (double)tri[5 * k + 5];
  if (blockIdx.x == 0)
    for (int i = threadIdx.x; i < k; i += blockDim.x) lam_out[i] = (double)tri[4 * k + i] * hmax;
  const int lane = threadIdx.x & 31;
  const int c = blockIdx.x * 8 + (threadIdx.x >> 5);
  if (c >= k) return;
  float z[4];
#pragma unroll
  for (int t = 0; t < 4; ++t) {
    const int r = lane + 32 * t;
    z[t] = r < k ? gZ[r * k + c] : 0.f;
  }
  for (int j = k - 3; j >= 0; --j) {
    const float b = beta[j];
    if (b == 0.f) continue;  // uniform across the warp
    float v[4], dot = 0.f;
#pragma unroll
    for (int t = 0; t < 4; ++t) {
      const int r = lane + 32 * t;
      v[t] = r < k ? Vs[j * k + r] : 0.f;
      dot = fmaf(v[t], z[t], dot);
    }
    const float w = b * warp_sumf(dot);
#pragma unroll
    for (int t = 0; t < 4; ++t) z[t] = fmaf(-w, v[t], z[t]);
  }
#pragma unroll
  for (int t = 0; t < 4; ++t) {
    const int r = lane + 32 * t;
    if (r < k) Xout[r * k + c] = (double)z[t];
  }
}

void launch_eig_seed(Launcher& L, const double* H, int k, float* gA, float* gZ, float* gQ, float* tri, double* Xout,
                     double* lam, double* scal, int32_t* nclusters) {
  if (k <= 128) {
    const size_t s1 = (size_t)128 * k * sizeof(float);
    cudaFuncSetAttribute(seed_tri_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)s1);
    seed_tri_kernel<<<1, kSeedThreads, s1, L.stream>>>(H, k, gA, tri, scal);
    seed_bisect_kernel<<<(k + 3) / 4, 128, 0, L.stream>>>(k, tri);
    const size_t s3 = (size_t)2 * k * k * sizeof(float);
    cudaFuncSetAttribute(seed_vec_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)s3);
    seed_vec_kernel<<<1, 128, s3, L.stream>>>(k, tri, gZ, nclusters);
    const size_t s4 = (size_t)k * k * sizeof(float);
    cudaFuncSetAttribute(seed_back_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)s4);
    seed_back_kernel<<<(k + 7) / 8, 256, s4, L.stream>>>(k, gA, gZ, tri, Xout, lam);
    L.count(4);
    return;
  }
  eig_seed_kernel<<<1, kSeedThreads, 0, L.stream>>>(H, k, gA, gZ, gQ, Xout, lam, scal, nclusters);
  L.count(1);
}

}  // namespace lspca
