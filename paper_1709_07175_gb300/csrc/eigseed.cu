// FP32 seed of the symmetric eigensolve of the k x k step (k <= 256), one
// level of a graded solve.
//
// The eigen route of the table footnote (Sec. III) squares the singular
// values of F = U^T X, so the eigenvalues of H = F F^T span the fourth power
// of the spectrum of X: on uncentred binary features the first is 10^4 to
// 10^5 times the rest, and a decaying spectrum puts most eigenvalues far
// below FP32 resolution of the largest.  An FP32 seed of the whole H cannot
// separate those.  The solve is therefore graded (small.cu drives it):
//   level 0   seeds H;  eigenvalues below kTailTau times the largest form the
//             "tail" and get only an orthonormal basis of their subspace;
//   level l   after the FP64 refinement of level l - 1, seeds the leading
//             block S[0:t, 0:t] of S = W^T H W over that tail (t columns,
//             a prefix in ascending order), scaled by its own largest entry,
//             so FP32 resolves the next four decades; its vectors rotate the
//             tail columns of W.
// Block sizes live on the device (lvl[l]), so the launch sequence is fixed
// and a level whose block has fewer than two columns does nothing.
//
// One level of the seed, on the s x s block (s <= 256), scaled by 1/max|M_ii|:
//   1. Householder tridiagonalisation M = Q T Q^T on one CTA:
//      seed_tri_col_kernel for k <= 128 (each column in the registers of a
//      thread pair, two block barriers per step, the next reflector formed
//      by one warp during the update); seed_tri_kernel above (thread (g, c)
//      owns column c and rows g + 4i; rows below 128 in registers, the rest
//      in shared memory; every thread derives the reflector of step j from
//      row j, published by its owners with per-warp partial norms; three
//      block barriers per step).
//   2. seed_bisect_kernel: one warp per eigenvalue, Sturm counts at 32
//      interior points per round, 6 rounds (33^6 >= 2^30: the resolution of
//      30 halvings of the Gershgorin interval).
//   3. seed_ii_kernel: one thread per eigenvalue outside the tail, two steps
//      of inverse iteration with an LDL^T solve of T - lambda I.
//   4. seed_orth_kernel (one CTA): eigenvalues closer than kClusterTol ||T||
//      form clusters; each cluster's vectors are replaced by an orthonormal
//      basis of their span (Householder QR), and the tail gets an
//      orthonormal basis of the complement of the other vectors (the
//      trailing columns of the Q factor of their Householder QR).  The cost
//      is one QR step per clustered vector, plus one per non-tail vector when
//      there is a tail.
//   5. seed_back_kernel: W = Q Z, one warp per column.
#include "common.cuh"
#include "kernels.h"

namespace lspca {

constexpr float kTailTau = 1e-4f;     // tail: eigenvalues below this times the largest of the level
constexpr float kClusterTol = 1e-5f;  // cluster: consecutive eigenvalues closer than this times ||T||

// Layout of `tri` (floats), for a k-wide workspace:
//   d [0, k), e [k, 2k), e^2 [2k, 3k), beta [3k, 4k), eigenvalues of T
//   (ascending) [4k, 5k), then gl, gu, ||T||, pivmin, max|M_ii| as hi + lo.
__device__ __forceinline__ int level_size(const int32_t* lvl, int level, int k) { return level == 0 ? k : lvl[level]; }

// Number of eigenvalues of T (d, e) smaller than x (Sturm count).
__device__ __forceinline__ int sturm_count(const float* d, const float* e2, int s, float x, float pivmin) {
  int c = 0;
  float q = d[0] - x;
  if (fabsf(q) < pivmin) q = -pivmin;
  c += q < 0.f;
  for (int i = 1; i < s; ++i) {
    q = d[i] - x - __fdividef(e2[i - 1], q);
    if (fabsf(q) < pivmin) q = -pivmin;
    c += q < 0.f;
  }
  return c;
}

// ---------------------------------------------------------------------------
// 1. Tridiagonalisation.
template <int NC>
struct TriCfg {
  static constexpr int THREADS = 4 * NC;
  static constexpr int NR = NC / 4;              // rows per thread
  static constexpr int NRR = NR < 32 ? NR : 32;  // of them in registers (rows < 128)
  static constexpr int NRS = NR - NRR;           // in shared memory (rows 128 .. NC-1)
  static constexpr int NW = THREADS / 32;
  static constexpr int GW = NC / 32;             // warps per row group
  // floats of dynamic shared memory
  static constexpr int SMEM_FLOATS = NRS * 4 * NC   // rows >= 128
                                     + 2 * NC       // row j, natural order (ping-pong)
                                     + 2 * NC       // x of row j, permuted (ping-pong)
                                     + NC           // w, permuted
                                     + 4 * NC       // partial matrix-vector products
                                     + NW           // partial v^T A v
                                     + 2 * 8        // partial squared norms (ping-pong)
                                     + 3 * NC;      // d, e, beta
};

__device__ __forceinline__ int perm_of(int r, int nr) { return (r & 3) * nr + (r >> 2); }

// Reflector j of the tridiagonalisation has entries in rows j+1 .. s-1; they
// are stored packed, reflector after reflector.
__device__ __forceinline__ int packed_off(int j, int s) { return j * (s - 1) - j * (j - 1) / 2; }

template <int NC>
__global__ void __launch_bounds__(4 * NC, 1) seed_tri_kernel(const double* __restrict__ M, int k, int level,
                                                            int32_t* lvl, float* __restrict__ gV,
                                                            float* __restrict__ tri, double* scal) {
  pdl_wait();  // first, on every path: completion stays ordered along the chain
  using C = TriCfg<NC>;
  constexpr int NR = C::NR, NRR = C::NRR, NRS = C::NRS, GW = C::GW;
  extern __shared__ __align__(16) float sm[];
  float* As = sm;                           // (r - 128) * NC + c
  float* rowb = As + NRS * 4 * NC;          // [2][NC]
  float* rowp = rowb + 2 * NC;              // [2][NC] permuted, x_r = A[j][r] for r > j, else 0
  float* wp = rowp + 2 * NC;                // [NC] permuted w
  float* gpart = wp + NC;                   // [4][NC]
  float* vavp = gpart + 4 * NC;             // [NW]
  float* sqp = vavp + C::NW;                // [2][8]
  float* dv = sqp + 16;                     // [NC]
  float* ev = dv + NC;                      // [NC]
  float* bv = ev + NC;                      // [NC]
  __shared__ double red[32];
  __shared__ double hmax_s;

  const int s = level_size(lvl, level, k);
  if (level > 0 && s < 2) return;  // uniform: nothing to resolve at this level
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int c = tid % NC, g = tid / NC;
  const int cw0 = (warp % GW) * 32;  // first column of this warp
  if (level == 0 && tid < 3) lvl[1 + tid] = 0;

  // scale by 1 / max |M_ii| over the block; ||H||_F at level 0 (refinement noise floor)
  {
    double mx = 0.0;
    for (int i = tid; i < s; i += C::THREADS) mx = fmax(mx, fabs(M[(int64_t)i * k + i]));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if (lane == 0) red[warp] = mx;
    __syncthreads();
    if (tid == 0) {
      double m2 = 0.0;
      for (int i = 0; i < C::NW; ++i) m2 = fmax(m2, red[i]);
      hmax_s = m2 > 0.0 ? m2 : 1.0;
    }
    __syncthreads();
    if (level == 0) {
      double hf = 0.0;
      for (int e = tid; e < s * s; e += C::THREADS) {
        const double h = M[(int64_t)(e / s) * k + (e % s)];
        hf += h * h;
      }
      hf = warp_sum(hf);
      __syncthreads();
      if (lane == 0) red[warp] = hf;
      __syncthreads();
      if (tid == 0) {
        double sum = 0.0;
        for (int i = 0; i < C::NW; ++i) sum += red[i];
        scal[1] = sqrt(sum);
      }
    }
  }
  const double sc = 1.0 / hmax_s;
  float a[NRR];
#pragma unroll
  for (int i = 0; i < NRR; ++i) {
    const int r = g + 4 * i;
    a[i] = (r < s && c < s) ? (float)(M[(int64_t)r * k + c] * sc) : 0.f;
  }
#pragma unroll 4
  for (int i = NRR; i < NR; ++i) {
    const int r = g + 4 * i;
    As[(r - 128) * NC + c] = (r < s && c < s) ? (float)(M[(int64_t)r * k + c] * sc) : 0.f;
  }
  for (int e = tid; e < 2 * NC; e += C::THREADS) rowp[e] = 0.f;
  // value of A[row][c] held by this thread (row owned by group g; dynamic row)
  auto get_own = [&](int row) -> float {
    const int i = row >> 2;
    if (i >= NRR) return As[(row - 128) * NC + c];
    float v = 0.f;
#pragma unroll
    for (int q = 0; q < NRR; ++q)
      if (q == i) v = a[q];
    return v;
  };
  // publish row `row` (owners: group row & 3) into ping-pong buffer b: natural
  // order, the permuted x (entries right of row + 1... i.e. columns > row, as
  // the next reflector's x), and per-warp partial norms of columns > row + 1
  auto publish = [&](int row, int b, float val) {
    rowb[b * NC + c] = val;
    const float xv = (c > row && c < s) ? val : 0.f;
    rowp[b * NC + perm_of(c, NR)] = xv;
    float q = (c > row + 1 && c < s) ? val * val : 0.f;
    q = warp_sumf(q);
    if (lane == 0) sqp[b * 8 + (warp % GW)] = q;
  };
  __syncthreads();
  if (g == 0) publish(0, 0, a[0]);
  __syncthreads();

  for (int j = 0; j + 2 < s; ++j) {
    const int b = j & 1;
    const float* rb = rowb + b * NC;
    const float* rp = rowp + b * NC;
    // ---- phase 1: reflector (every thread, same data), partial A' u.  The
    // reflector is kept as a unit vector u = v / |v| (H = I - 2 u u^T), and the
    // row is scaled by 1 / |v| as it is loaded, so no product of the step
    // over- or underflows however small the row is; a row below 1e-18 of the
    // scaled block is taken as reduced.
    float sq = 0.f;
#pragma unroll
    for (int w = 0; w < GW; ++w) sq += sqp[b * 8 + w];
    const float x0 = rb[j + 1];
    const float nrm = sqrtf(x0 * x0 + sq);
    float alpha = 0.f, invv = 0.f;
    if (nrm > 1e-18f) {
      alpha = x0 >= 0.f ? -nrm : nrm;
      const float v0 = x0 - alpha;
      invv = rsqrtf(v0 * v0 + sq);
    }
    const bool refl = invv > 0.f;
    if (tid == 0) {
      dv[j] = rb[j];
      ev[j] = refl ? alpha : x0;
      bv[j] = refl ? 2.f : 0.f;
    }
    const int own = (j + 1) & 3;
    const bool wact = (cw0 + 31 > j) && (cw0 < s);  // warp holds an active column
    // u_c of the own column: u = (x - alpha e_{j+1}) / |v|
    const float uc = (c > j && c < s) ? (rb[c] - (c == j + 1 ? alpha : 0.f)) * invv : 0.f;
    if (g == 0 && c > j && c < s) gV[packed_off(j, s) + (c - j - 1)] = uc;
    if (!refl) {
      // nothing to reduce: publish row j + 1 unchanged
      __syncthreads();
      if (g == own) publish(j + 1, b ^ 1, get_own(j + 1));
      __syncthreads();
      continue;
    }
    float pc = 0.f;
    if (wact) {
      // row groups of four (rows g + 4i .. g + 4i + 12) wholly at or above row
      // j hold x = 0 and are skipped (uniform per warp)
      const float4* xp = reinterpret_cast<const float4*>(rp + g * NR);
      if (j < 127) {
#pragma unroll
        for (int i = 0; i < NRR; i += 4) {
          if (g + 4 * (i + 3) <= j) continue;
          const float4 x = xp[i / 4];
          pc = fmaf(a[i], x.x, pc);
          pc = fmaf(a[i + 1], x.y, pc);
          pc = fmaf(a[i + 2], x.z, pc);
          pc = fmaf(a[i + 3], x.w, pc);
        }
      }
      const int is = j < 128 ? NRR : max(NRR, ((j - g) >> 2) & ~3);
#pragma unroll 4
      for (int i = is; i < NR; i += 4) {
        const float4 x = xp[i / 4];
        const float* ar = As + (g + 4 * i - 128) * NC + c;
        pc = fmaf(ar[0], x.x, pc);
        pc = fmaf(ar[4 * NC], x.y, pc);
        pc = fmaf(ar[8 * NC], x.z, pc);
        pc = fmaf(ar[12 * NC], x.w, pc);
      }
      if (g == own) pc = fmaf(-alpha, get_own(j + 1), pc);  // the -alpha e_{j+1} part of v
      pc *= invv;                                            // A' u = A' v / |v|
    }
    gpart[g * NC + c] = pc;
    {
      float t = uc * pc;
      t = warp_sumf(t);
      if (lane == 0) vavp[warp] = t;
    }
    __syncthreads();
    // ---- phase 2: q = A' u, p = 2 q, K = 2 u^T q, w = p - K u
    float uau = 0.f;
#pragma unroll
    for (int w = 0; w < C::NW; w += 4) {
      const float4 t = *reinterpret_cast<const float4*>(vavp + w);
      uau += (t.x + t.y) + (t.z + t.w);
    }
    const float K = 2.f * uau;
    const float p = 2.f * ((gpart[c] + gpart[NC + c]) + (gpart[2 * NC + c] + gpart[3 * NC + c]));
    const float wc = (c > j && c < s) ? p - K * uc : 0.f;
    if (g == 0) wp[perm_of(c, NR)] = wc;
    __syncthreads();
    // ---- phase 3: A' -= u w^T + w u^T (rows through x / |v|, row j + 1
    // corrected by alpha w / |v|), then the owners publish row j + 1
    if (wact) {
      const float4* xp = reinterpret_cast<const float4*>(rp + g * NR);
      const float4* wq = reinterpret_cast<const float4*>(wp + g * NR);
      const float wci = wc * invv;
      if (j < 127) {
#pragma unroll
        for (int i = 0; i < NRR; i += 4) {
          if (g + 4 * (i + 3) <= j) continue;
          const float4 x = xp[i / 4], w = wq[i / 4];
          a[i] -= fmaf(x.x, wci, w.x * uc);
          a[i + 1] -= fmaf(x.y, wci, w.y * uc);
          a[i + 2] -= fmaf(x.z, wci, w.z * uc);
          a[i + 3] -= fmaf(x.w, wci, w.w * uc);
        }
      }
      const int is = j < 128 ? NRR : max(NRR, ((j - g) >> 2) & ~3);
#pragma unroll 4
      for (int i = is; i < NR; i += 4) {
        const float4 x = xp[i / 4], w = wq[i / 4];
        float* ar = As + (g + 4 * i - 128) * NC + c;
        ar[0] -= fmaf(x.x, wci, w.x * uc);
        ar[4 * NC] -= fmaf(x.y, wci, w.y * uc);
        ar[8 * NC] -= fmaf(x.z, wci, w.z * uc);
        ar[12 * NC] -= fmaf(x.w, wci, w.w * uc);
      }
    }
    if (g == own) {
      // row j + 1: add alpha w_c / |v| back (the row update above used x_{j+1}, not v_{j+1})
      const int i1 = (j + 1) >> 2;
      const float corr = alpha * invv * wc;
      float val;
      if (i1 >= NRR) {
        float* ar = As + (j + 1 - 128) * NC + c;
        if (wact) *ar += corr;
        val = *ar;
      } else {
        val = 0.f;
#pragma unroll
        for (int q = 0; q < NRR; ++q)
          if (q == i1) {
            if (wact) a[q] += corr;
            val = a[q];
          }
      }
      publish(j + 1, b ^ 1, val);
    }
    __syncthreads();
  }
  // the last 2 x 2 block (rows s-2, s-1), or the 1 x 1 matrix
  if (s >= 2) {
    const int bl = (s - 2) & 1;  // row s-2 was published last (row 0 when s == 2)
    if (tid == 0) {
      dv[s - 2] = rowb[bl * NC + s - 2];
      ev[s - 2] = rowb[bl * NC + s - 1];
      bv[s - 2] = 0.f;
      bv[s - 1] = 0.f;
    }
    if (g == ((s - 1) & 3) && c == s - 1) dv[s - 1] = get_own(s - 1);
  } else if (tid == 0) {
    dv[0] = a[0];
    bv[0] = 0.f;
  }
  __syncthreads();
  for (int i = tid; i < s; i += C::THREADS) {
    tri[i] = dv[i];
    tri[k + i] = (i + 1 < s) ? ev[i] : 0.f;
    tri[2 * k + i] = (i + 1 < s) ? ev[i] * ev[i] : 0.f;
    tri[3 * k + i] = bv[i];
  }
  if (tid == 0) {
    float gl = 1e30f, gu = -1e30f, tn = 0.f;
    for (int i = 0; i < s; ++i) {
      const float off = (i > 0 ? fabsf(ev[i - 1]) : 0.f) + (i + 1 < s ? fabsf(ev[i]) : 0.f);
      gl = fminf(gl, dv[i] - off);
      gu = fmaxf(gu, dv[i] + off);
      tn = fmaxf(tn, fabsf(dv[i]) + off);
    }
    const float pad = 2.f * 1.2e-7f * tn + 1e-30f;
    float* cst = tri + 5 * k;
    cst[0] = gl - pad;
    cst[1] = gu + pad;
    cst[2] = tn;
    cst[3] = fmaxf(1e-30f, 1.2e-7f * 1e-6f * tn);  // pivmin
    const float hi = (float)hmax_s;
    cst[4] = hi;
    cst[5] = (float)(hmax_s - (double)hi);
  }
}

// Tridiagonalisation for blocks of at most 128 (k <= 128), the columns held
// in registers: thread t owns column c = t / 2 and, of its row groups of four,
// those of parity h = t & 1 (rows 8 i + 4 h .. 8 i + 4 h + 3).  A stays
// symmetric under the two-sided update, so the next reflector's source row
// j + 1 is column j + 1, and no register is ever indexed at run time.  Per
// step j: q = A u over the active columns (u = v / |v|, v the Householder
// vector with the rows at or above j zeroed), the block sum K = 2 u^T q, and
// the rank-2 update A -= u w^T + w u^T (w = 2 q - K u) written as
// a -= v_r al_c + q_r be_c, so only q and K are exchanged: two block
// barriers.  Warp 0 forms the next step's reflector (norm, alpha, masked v)
// from column j + 1 as it was before the step -- stored one step ahead by
// its owners -- plus this step's update, while the other warps apply it.
// Outputs are those of seed_tri_kernel.
constexpr int kTC = 256;

__global__ void __launch_bounds__(kTC, 1) seed_tri_col_kernel(const double* __restrict__ M, int k, int level,
                                                              int32_t* lvl, float* __restrict__ gV,
                                                              float* __restrict__ tri, double* scal) {
  pdl_wait();  // first, on every path: completion stays ordered along the chain
  __shared__ __align__(16) float xs[2][128];  // v of the step (ping-pong)
  __shared__ __align__(16) float qs[128];     // q = A u of the step
  __shared__ __align__(16) float cs[2][128];  // lookahead column (ping-pong)
  __shared__ float invv_s[2];
  __shared__ float red[8];
  __shared__ float dv[128], ev[128], bv[128];
  __shared__ double redd[8];
  __shared__ double hmax_s;

  const int s = level_size(lvl, level, k);
  if (level > 0 && s < 2) return;  // uniform: nothing to resolve at this level
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int c = tid >> 1, h = tid & 1;
  if (level == 0 && tid < 3) lvl[1 + tid] = 0;

  // scale by 1 / max |M_ii| over the block; ||H||_F at level 0 (refinement noise floor)
  {
    double mx = 0.0;
    for (int i = tid; i < s; i += kTC) mx = fmax(mx, fabs(M[(int64_t)i * k + i]));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if (lane == 0) redd[warp] = mx;
    __syncthreads();
    if (tid == 0) {
      double m2 = 0.0;
      for (int i = 0; i < kTC / 32; ++i) m2 = fmax(m2, redd[i]);
      hmax_s = m2 > 0.0 ? m2 : 1.0;
    }
    __syncthreads();
    if (level == 0) {
      double hf = 0.0;
      for (int e = tid; e < s * s; e += kTC) {
        const double v = M[(int64_t)(e / s) * k + (e % s)];
        hf += v * v;
      }
      hf = warp_sum(hf);
      if (lane == 0) redd[warp] = hf;
      __syncthreads();
      if (tid == 0) {
        double sum = 0.0;
        for (int i = 0; i < kTC / 32; ++i) sum += redd[i];
        scal[1] = sqrt(sum);
      }
    }
  }
  const double sc = 1.0 / hmax_s;
  float a[16][4];
#pragma unroll
  for (int i = 0; i < 16; ++i)
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const int r = 8 * i + 4 * h + e;
      a[i][e] = (r < s && c < s) ? (float)(M[(int64_t)r * k + c] * sc) : 0.f;
    }
  auto store_col = [&](float* dst) {
#pragma unroll
    for (int i = 0; i < 16; ++i)
      *reinterpret_cast<float4*>(dst + 8 * i + 4 * h) = make_float4(a[i][0], a[i][1], a[i][2], a[i][3]);
  };
  // reflector of step jn from column jn (all lanes of the warp owning it)
  auto prepare = [&](int jn, int b) {
    float* x = xs[b];
    if (c == jn) store_col(x);
    __syncwarp();
    const float4 x4 = *reinterpret_cast<const float4*>(x + 4 * lane);
    const float x0 = x[jn + 1], dj = x[jn];
    const float xe[4] = {x4.x, x4.y, x4.z, x4.w};
    float sq = 0.f;
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const int r = 4 * lane + e;
      if (r > jn + 1 && r < s) sq = fmaf(xe[e], xe[e], sq);
    }
    sq = warp_sumf(sq);
    // the reflector as a unit vector u = v / |v|; a column below 1e-18 of the
    // scaled block is taken as reduced (u = 0)
    const float nrm = sqrtf(x0 * x0 + sq);
    float alpha = 0.f, invv = 0.f;
    if (nrm > 1e-18f) {
      alpha = x0 >= 0.f ? -nrm : nrm;
      const float v0 = x0 - alpha;
      invv = rsqrtf(v0 * v0 + sq);
    }
    __syncwarp();  // every lane has read x before it is masked
    float m[4];
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const int r = 4 * lane + e;
      m[e] = r <= jn ? 0.f : (r == jn + 1 ? x0 - alpha : xe[e]);
    }
    *reinterpret_cast<float4*>(x + 4 * lane) = make_float4(m[0], m[1], m[2], m[3]);
    if (lane == 0) {
      invv_s[b] = invv;
      dv[jn] = dj;
      ev[jn] = invv > 0.f ? alpha : x0;
      bv[jn] = invv > 0.f ? 2.f : 0.f;
    }
  };
  // before step 0: its reflector from column 0, and column 1 for the lookahead
  if (warp == 0) {
    if (s >= 3) prepare(0, 0);
    if (s >= 4 && c == 1) store_col(cs[0]);
  }
  __syncthreads();

  for (int j = 0; j + 2 < s; ++j) {
    const int b = j & 1;
    const float* x = xs[b];
    const float invv = invv_s[b];
    const bool act = c > j && c < s;
    // q_c = (A u)_c; the column pair adds its two halves.  Rows go in
    // segments of 32 (four groups per thread), skipped when they lie at or
    // above j; warps whose columns are all finished skip the products (both
    // tests are uniform over the warp; inactive lanes of an active warp
    // compute values that are never used)
    const bool wact = (16 * warp + 15 > j) && (16 * warp < s);
    float pc = 0.f;
    if (wact) {
      float p0 = 0.f, p1 = 0.f, p2 = 0.f, p3 = 0.f;
#pragma unroll
      for (int sg = 0; sg < 4; ++sg) {
        if (32 * sg + 31 <= j) continue;
#pragma unroll
        for (int ii = 0; ii < 4; ++ii) {
          const int i = 4 * sg + ii;
          const float4 v = *reinterpret_cast<const float4*>(x + 8 * i + 4 * h);
          p0 = fmaf(a[i][0], v.x, p0);
          p1 = fmaf(a[i][1], v.y, p1);
          p2 = fmaf(a[i][2], v.z, p2);
          p3 = fmaf(a[i][3], v.w, p3);
        }
      }
      pc = act ? (p0 + p1) + (p2 + p3) : 0.f;
    }
    pc += __shfl_xor_sync(0xffffffffu, pc, 1);
    const float q = pc * invv;
    const float uc = act ? x[c] * invv : 0.f;
    if (h == 0) {
      qs[c] = q;  // zero for finished and padding columns
      if (act) gV[packed_off(j, s) + (c - j - 1)] = uc;
    }
    const float t = warp_sumf((h == 0 && act) ? uc * q : 0.f);
    if (lane == 0) red[warp] = t;
    __syncthreads();
    // K = 2 u^T q, w = 2 q - K u.  A -= u w^T + w u^T is, entry by entry,
    // a -= v_r al_c + q_r be_c with al_c = (w_c - K u_c) / |v|, be_c = 2 u_c
    // (rows at or above j and padding rows have v = q = 0)
    float uau = 0.f;
#pragma unroll
    for (int w = 0; w < kTC / 32; ++w) uau += red[w];
    const float K = 2.f * uau;
    if (wact) {
      const float al = invv * (2.f * q - 2.f * K * uc), be = 2.f * uc;
#pragma unroll
      for (int sg = 0; sg < 4; ++sg) {
        if (32 * sg + 31 <= j) continue;
#pragma unroll
        for (int ii = 0; ii < 4; ++ii) {
          const int i = 4 * sg + ii;
          const float4 v = *reinterpret_cast<const float4*>(x + 8 * i + 4 * h);
          const float4 w = *reinterpret_cast<const float4*>(qs + 8 * i + 4 * h);
          a[i][0] = fmaf(-v.x, al, fmaf(-w.x, be, a[i][0]));
          a[i][1] = fmaf(-v.y, al, fmaf(-w.y, be, a[i][1]));
          a[i][2] = fmaf(-v.z, al, fmaf(-w.z, be, a[i][2]));
          a[i][3] = fmaf(-v.w, al, fmaf(-w.w, be, a[i][3]));
        }
      }
    }
    // column j + 2 (now as after step j) for the next step's lookahead
    if (c == j + 2 && j + 2 < s) store_col(cs[(j + 1) & 1]);
    // warp 0: the reflector of step j + 1 from column j + 1 as before this
    // step plus this step's update, while the other warps update
    if (warp == 0 && j + 3 < s) {
      const int jn = j + 1, bn = b ^ 1;
      const float* cp = cs[b];
      const float un = x[jn] * invv, qn = qs[jn];
      const float aln = invv * (2.f * qn - 2.f * K * un), ben = 2.f * un;
      const float4 c4 = *reinterpret_cast<const float4*>(cp + 4 * lane);
      const float4 v4 = *reinterpret_cast<const float4*>(x + 4 * lane);
      const float4 q4 = *reinterpret_cast<const float4*>(qs + 4 * lane);
      const float xe[4] = {fmaf(-v4.x, aln, fmaf(-q4.x, ben, c4.x)), fmaf(-v4.y, aln, fmaf(-q4.y, ben, c4.y)),
                           fmaf(-v4.z, aln, fmaf(-q4.z, ben, c4.z)), fmaf(-v4.w, aln, fmaf(-q4.w, ben, c4.w))};
      const float x0 = fmaf(-x[jn + 1], aln, fmaf(-qs[jn + 1], ben, cp[jn + 1]));
      const float dj = fmaf(-x[jn], aln, fmaf(-qn, ben, cp[jn]));
      float sq = 0.f;
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const int r = 4 * lane + e;
        if (r > jn + 1 && r < s) sq = fmaf(xe[e], xe[e], sq);
      }
      sq = warp_sumf(sq);
      const float nrm = sqrtf(x0 * x0 + sq);
      float alpha = 0.f, iv = 0.f;
      if (nrm > 1e-18f) {
        alpha = x0 >= 0.f ? -nrm : nrm;
        const float v0 = x0 - alpha;
        iv = rsqrtf(v0 * v0 + sq);
      }
      float m[4];
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const int r = 4 * lane + e;
        m[e] = r <= jn ? 0.f : (r == jn + 1 ? x0 - alpha : xe[e]);
      }
      *reinterpret_cast<float4*>(xs[bn] + 4 * lane) = make_float4(m[0], m[1], m[2], m[3]);
      if (lane == 0) {
        invv_s[bn] = iv;
        dv[jn] = dj;
        ev[jn] = iv > 0.f ? alpha : x0;
        bv[jn] = iv > 0.f ? 2.f : 0.f;
      }
    }
    __syncthreads();
  }
  // the last 2 x 2 block (rows s-2, s-1), or the 1 x 1 matrix
  if (s >= 2) {
    if (c == s - 2) store_col(xs[0]);
    if (c == s - 1) store_col(xs[1]);
  } else if (c == 0) {
    store_col(xs[1]);
  }
  __syncthreads();
  if (tid == 0) {
    if (s >= 2) {
      dv[s - 2] = xs[0][s - 2];
      ev[s - 2] = xs[0][s - 1];
      dv[s - 1] = xs[1][s - 1];
      bv[s - 2] = 0.f;
      bv[s - 1] = 0.f;
    } else {
      dv[0] = xs[1][0];
      bv[0] = 0.f;
    }
  }
  __syncthreads();
  for (int i = tid; i < s; i += kTC) {
    tri[i] = dv[i];
    tri[k + i] = (i + 1 < s) ? ev[i] : 0.f;
    tri[2 * k + i] = (i + 1 < s) ? ev[i] * ev[i] : 0.f;
    tri[3 * k + i] = bv[i];
  }
  if (tid == 0) {
    float gl = 1e30f, gu = -1e30f, tn = 0.f;
    for (int i = 0; i < s; ++i) {
      const float off = (i > 0 ? fabsf(ev[i - 1]) : 0.f) + (i + 1 < s ? fabsf(ev[i]) : 0.f);
      gl = fminf(gl, dv[i] - off);
      gu = fmaxf(gu, dv[i] + off);
      tn = fmaxf(tn, fabsf(dv[i]) + off);
    }
    const float pad = 2.f * 1.2e-7f * tn + 1e-30f;
    float* cst = tri + 5 * k;
    cst[0] = gl - pad;
    cst[1] = gu + pad;
    cst[2] = tn;
    cst[3] = fmaxf(1e-30f, 1.2e-7f * 1e-6f * tn);  // pivmin
    const float hi = (float)hmax_s;
    cst[4] = hi;
    cst[5] = (float)(hmax_s - (double)hi);
  }
}

// ---------------------------------------------------------------------------
// 2. Eigenvalues of T, ascending: one warp per eigenvalue idx.
__global__ void __launch_bounds__(128) seed_bisect_kernel(int k, int level, const int32_t* __restrict__ lvl,
                                                          float* tri) {
  pdl_wait();  // first, on every path: completion stays ordered along the chain
  const int s = level_size(lvl, level, k);
  if (level > 0 && s < 2) return;
  __shared__ float d[256], e2[256];
  for (int i = threadIdx.x; i < s; i += blockDim.x) {
    d[i] = tri[i];
    e2[i] = tri[2 * k + i];
  }
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const int idx = blockIdx.x * 4 + (threadIdx.x >> 5);
  if (idx >= s) return;
  const float* cst = tri + 5 * k;
  const float pivmin = cst[3];
  float lo = cst[0], hi = cst[1];
#pragma unroll 1
  for (int it = 0; it < 6; ++it) {
    const float x = lo + (hi - lo) * (float)(lane + 1) / 33.f;
    const bool above = sturm_count(d, e2, s, x, pivmin) > idx;
    const unsigned ball = __ballot_sync(0xffffffffu, above);
    const int first = ball ? __ffs((int)ball) - 1 : 32;  // first point with count > idx
    const float nlo = first == 0 ? lo : lo + (hi - lo) * (float)first / 33.f;
    const float nhi = first == 32 ? hi : lo + (hi - lo) * (float)(first + 1) / 33.f;
    lo = nlo;
    hi = nhi;
  }
  if (lane == 0) tri[4 * k + idx] = 0.5f * (lo + hi);
}

// Tail size of a level: the eigenvalues below kTailTau times the largest (a
// prefix of the ascending list); a tail of one is resolved like the others.
__device__ __forceinline__ int tail_count(const float* lam, int s) {
  const float lim = kTailTau * lam[s - 1];
  int t = 0;
  while (t < s && lam[t] < lim) ++t;
  return t >= 2 ? t : 0;
}

// ---------------------------------------------------------------------------
// 3. Inverse iteration, one thread per eigenvalue outside the tail, 32 per
// CTA; each thread's vector and pivots live in shared memory (row r of the
// CTA's vectors at r * 33: conflict-free for the threads and for the
// coalesced copy out).  Zc is column-major (vector i at Zc[i k ...]).
constexpr int kIIThreads = 32;

__global__ void __launch_bounds__(kIIThreads) seed_ii_kernel(int k, int level, const int32_t* __restrict__ lvl,
                                                             const float* __restrict__ tri, float* __restrict__ Zc) {
  pdl_wait();  // first, on every path: completion stays ordered along the chain
  const int s = level_size(lvl, level, k);
  if (level > 0 && s < 2) return;
  extern __shared__ float zsm[];
  float* zs = zsm;              // s x 33
  float* qs = zsm + 33 * 256;   // s x 33
  __shared__ float d[256], e[256], lam[256];
  const int lane = threadIdx.x;
  for (int i = lane; i < s; i += kIIThreads) {
    d[i] = tri[i];
    e[i] = tri[k + i];
    lam[i] = tri[4 * k + i];
  }
  __syncwarp();
  const int tcount = tail_count(lam, s);
  const int i0 = blockIdx.x * kIIThreads;
  if (i0 + kIIThreads <= tcount || i0 >= s) return;  // uniform: no vector of this CTA is computed
  const int i = i0 + lane;
  const bool mine = i < s && i >= tcount;
  const float pivmin = tri[5 * k + 3];
  if (mine) {
    const float mu = lam[i];
    float* z = zs + lane;
    float* q = qs + lane;
    for (int r = 0; r < s; ++r) z[r * 33] = 1.f + 0.5f * __sinf(0.7f * (float)(r + 3 * i) + 0.3f);
    for (int rep = 0; rep < 2; ++rep) {
      // LDL^T of T - mu I (tiny pivots replaced by -pivmin) fused with the
      // forward solve L y = z, then D L^T x = y and the normalisation
      float qi = d[0] - mu;
      if (fabsf(qi) < pivmin) qi = -pivmin;
      q[0] = qi;
      float y = z[0];
      for (int r = 1; r < s; ++r) {
        const float l = __fdividef(e[r - 1], qi);
        qi = d[r] - mu - l * e[r - 1];
        if (fabsf(qi) < pivmin) qi = -pivmin;
        q[r * 33] = qi;
        y = z[r * 33] - l * y;
        z[r * 33] = y;
      }
      float x = __fdividef(y, qi);
      z[(s - 1) * 33] = x;
      float nrm = x * x;
      for (int r = s - 2; r >= 0; --r) {
        const float rq = __fdividef(1.f, q[r * 33]);
        x = z[r * 33] * rq - (e[r] * rq) * x;
        z[r * 33] = x;
        nrm = fmaf(x, x, nrm);
      }
      if (!(nrm > 0.f) || !isfinite(nrm)) {  // overflow or a zero solve: a coordinate vector
        for (int r = 0; r < s; ++r) z[r * 33] = r == i ? 1.f : 0.f;
        break;
      }
      const float inv = rsqrtf(nrm);
      for (int r = 0; r < s; ++r) z[r * 33] *= inv;
    }
  }
  __syncwarp();
  // copy the computed vectors out, one vector per pass, lanes along rows
  for (int cc = 0; cc < kIIThreads; ++cc) {
    const int ic = i0 + cc;
    if (ic >= s || ic < tcount) continue;  // uniform
    for (int r = lane; r < s; r += kIIThreads) Zc[(int64_t)ic * k + r] = zs[r * 33 + cc];
  }
}

// ---------------------------------------------------------------------------
// 4. Orthonormal bases for clusters and the tail (one CTA of kOrthThreads).
constexpr int kOrthThreads = 1024;

// Householder QR of the nc columns src[0..nc) (column-major, length s, ld k)
// held in the working copy Wk (overwritten); reflector jj (rows jj..s-1) goes
// to U[jj k ...], its beta to bet[jj].  Two block barriers per column.
__device__ void hh_qr(float* Wk, int nc, int s, int k, float* U, float* bet) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int jj = 0; jj < nc; ++jj) {
    float* col = Wk + (int64_t)jj * k;
    if (warp == 0) {
      float sq = 0.f;
      for (int r = jj + 1 + lane; r < s; r += 32) sq = fmaf(col[r], col[r], sq);
      sq = warp_sumf(sq);
      const float x0 = col[jj];
      const float nrm = sqrtf(x0 * x0 + sq);
      float alpha = 0.f, beta = 0.f, u0 = x0;
      if (nrm > 1e-18f) {  // below that the column is taken as zero (no reflection)
        alpha = x0 >= 0.f ? -nrm : nrm;
        u0 = x0 - alpha;
        beta = 2.f / (u0 * u0 + sq);
      }
      float* u = U + (int64_t)jj * k;
      for (int r = lane; r < s; r += 32) u[r] = r < jj ? 0.f : (r == jj ? u0 : col[r]);
      if (lane == 0) bet[jj] = beta;
    }
    __syncthreads();
    const float beta = bet[jj];
    const float* u = U + (int64_t)jj * k;
    for (int cc = jj + 1 + warp; cc < nc; cc += nw) {
      float* z = Wk + (int64_t)cc * k;
      float dot = 0.f;
      for (int r = jj + lane; r < s; r += 32) dot = fmaf(u[r], z[r], dot);
      dot = beta * warp_sumf(dot);
      for (int r = jj + lane; r < s; r += 32) z[r] = fmaf(-dot, u[r], z[r]);
    }
    __syncthreads();
  }
}

// Column m of Q = H_0 H_1 ... H_{nc-1} (the reflectors of hh_qr) into dst
// (length s), one warp; lane holds rows lane + 32 t.
__device__ void hh_form_col(const float* U, const float* bet, int nc, int s, int k, int m, float* dst) {
  const int lane = threadIdx.x & 31;
  float y[8];
#pragma unroll
  for (int t = 0; t < 8; ++t) y[t] = (lane + 32 * t == m) ? 1.f : 0.f;
  for (int jj = nc - 1; jj >= 0; --jj) {
    const float beta = bet[jj];
    if (beta == 0.f) continue;
    const float* u = U + (int64_t)jj * k;
    float uv[8], dot = 0.f;
#pragma unroll
    for (int t = 0; t < 8; ++t) {
      const int r = lane + 32 * t;
      uv[t] = r < s ? u[r] : 0.f;
      dot = fmaf(uv[t], y[t], dot);
    }
    dot = beta * warp_sumf(dot);
#pragma unroll
    for (int t = 0; t < 8; ++t) y[t] = fmaf(-dot, uv[t], y[t]);
  }
#pragma unroll
  for (int t = 0; t < 8; ++t) {
    const int r = lane + 32 * t;
    if (r < s) dst[r] = y[t];
  }
}

__global__ void __launch_bounds__(kOrthThreads, 1) seed_orth_kernel(int k, int level, int32_t* lvl,
                                                                   const float* __restrict__ tri, float* Zc,
                                                                   float* U, float* Wk, int32_t* stats,
                                                                   int32_t* cid) {
  pdl_wait();  // first, on every path: completion stays ordered along the chain
  const int s = level_size(lvl, level, k);
  if (level > 0 && s < 2) return;
  __shared__ float lam[256];
  __shared__ float bet[256];
  __shared__ int cstart[257];
  __shared__ int ncl_s;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
  for (int i = tid; i < s; i += blockDim.x) lam[i] = tri[4 * k + i];
  __syncthreads();
  const int t = tail_count(lam, s);
  const float tol = kClusterTol * tri[5 * k + 2];
  if (tid == 0) {
    int nc = 0;
    for (int i = t; i < s; ++i)
      if (i == t || lam[i] - lam[i - 1] > tol) cstart[nc++] = i;
    cstart[nc] = s;
    ncl_s = nc;
    if (level + 1 < kSeedLevels) lvl[level + 1] = t;
    if (stats) *stats = level + 1;  // levels that ran
  }
  __syncthreads();
  const int ncl = ncl_s;
  // cluster ids of the block's columns: the tail is one cluster of the level
  for (int cl = 0; cl < ncl; ++cl)
    for (int i = cstart[cl] + tid; i < cstart[cl + 1]; i += blockDim.x) cid[i] = level * 1024 + cl;
  for (int i = tid; i < t; i += blockDim.x) cid[i] = level * 1024 + 1023;
  // clusters: Zc columns [i0, i1) <- orthonormal basis of their span.  The
  // vectors of a tight cluster come out of inverse iteration nearly parallel,
  // so their QR would bring rounding noise in from every direction: each is
  // first projected (twice) against the level's singleton vectors, which
  // span the rest of the block far more accurately.
  for (int cl = 0; cl < ncl; ++cl) {
    const int i0 = cstart[cl], i1 = cstart[cl + 1];
    const int nc = i1 - i0;
    if (nc < 2) continue;  // uniform
    for (int e = tid; e < nc * k; e += blockDim.x) Wk[e] = Zc[(int64_t)i0 * k + e];
    __syncthreads();
    for (int m = warp; m < nc; m += nw) {
      float* y = Wk + (int64_t)m * k;
      for (int pass = 0; pass < 2; ++pass)
        for (int sg = 0; sg < ncl; ++sg) {
          if (cstart[sg + 1] - cstart[sg] != 1) continue;  // singletons only
          const float* z = Zc + (int64_t)cstart[sg] * k;
          float dot = 0.f;
          for (int r = lane; r < s; r += 32) dot = fmaf(z[r], y[r], dot);
          dot = warp_sumf(dot);
          for (int r = lane; r < s; r += 32) y[r] = fmaf(-dot, z[r], y[r]);
        }
    }
    __syncthreads();
    hh_qr(Wk, nc, s, k, U, bet);
    for (int m = warp; m < nc; m += nw) hh_form_col(U, bet, nc, s, k, m, Zc + (int64_t)(i0 + m) * k);
    __syncthreads();
  }
  // tail: Zc columns [0, t) <- orthonormal basis of the complement of columns [t, s)
  if (t > 0) {
    const int r = s - t;
    for (int e = tid; e < r * k; e += blockDim.x) Wk[e] = Zc[(int64_t)t * k + e];
    __syncthreads();
    hh_qr(Wk, r, s, k, U, bet);
    for (int m = warp; m < t; m += nw) hh_form_col(U, bet, r, s, k, r + m, Zc + (int64_t)m * k);
  }
}

// ---------------------------------------------------------------------------
// 5. Back-transformation W = Q Z, one warp per column c of the k-wide output;
// the CTA stages the packed reflectors in shared memory.  Level 0: Xout = W
// (FP64 k x k, row-major) and lam_out = eigenvalues scaled back.  Level > 0:
// Xout = blockdiag(W, I_{k-s}).
constexpr int kBackWarps = 8;

__global__ void __launch_bounds__(kBackWarps * 32) seed_back_kernel(int k, int level, const int32_t* __restrict__ lvl,
                                                                    const float* __restrict__ gV,
                                                                    const float* __restrict__ Zc,
                                                                    const float* __restrict__ tri,
                                                                    double* __restrict__ Xout,
                                                                    double* __restrict__ lam_out) {
  pdl_wait();  // first, on every path: completion stays ordered along the chain
  const int s = level_size(lvl, level, k);
  if (level > 0 && s < 2) return;
  extern __shared__ __align__(16) float P[];  // packed reflectors
  __shared__ float bet[256];
  const int np = s >= 3 ? packed_off(s - 2, s) : 0;  // entries of reflectors 0 .. s-3
  for (int e = threadIdx.x; e < np; e += blockDim.x) P[e] = gV[e];
  for (int j = threadIdx.x; j < s; j += blockDim.x) bet[j] = tri[3 * k + j];
  __syncthreads();
  const double hmax = (double)tri[5 * k + 4] + (double)tri[5 * k + 5];
  if (level == 0 && blockIdx.x == 0)
    for (int i = threadIdx.x; i < s; i += blockDim.x) lam_out[i] = (double)tri[4 * k + i] * hmax;
  const int lane = threadIdx.x & 31;
  const int c = blockIdx.x * kBackWarps + (threadIdx.x >> 5);
  if (c >= k) return;
  if (c >= s) {  // identity outside the block (level > 0 only: s == k at level 0)
    for (int r = lane; r < k; r += 32) Xout[(int64_t)r * k + c] = r == c ? 1.0 : 0.0;
    return;
  }
  float z[8];
#pragma unroll
  for (int t = 0; t < 8; ++t) {
    const int r = lane + 32 * t;
    z[t] = r < s ? Zc[(int64_t)c * k + r] : 0.f;
  }
  for (int j = s - 3; j >= 0; --j) {
    const float b = bet[j];
    if (b == 0.f) continue;  // uniform across the warp
    const float* v = P + packed_off(j, s) - (j + 1);  // v[r], r in (j, s)
    float vv[8], dot = 0.f;
#pragma unroll
    for (int t = 0; t < 8; ++t) {
      const int r = lane + 32 * t;
      vv[t] = (r > j && r < s) ? v[r] : 0.f;
      dot = fmaf(vv[t], z[t], dot);
    }
    const float w = b * warp_sumf(dot);
#pragma unroll
    for (int t = 0; t < 8; ++t) z[t] = fmaf(-w, vv[t], z[t]);
  }
#pragma unroll
  for (int t = 0; t < 8; ++t) {
    const int r = lane + 32 * t;
    if (r < k) Xout[(int64_t)r * k + c] = r < s ? (double)z[t] : 0.0;
  }
}

template <int NC>
static void launch_tri(Launcher& L, const double* M, int k, int level, int32_t* lvl, float* gV, float* tri,
                       double* scal) {
  const size_t smem = (size_t)TriCfg<NC>::SMEM_FLOATS * sizeof(float);
  cudaFuncSetAttribute(seed_tri_kernel<NC>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  launch_pdl(L, seed_tri_kernel<NC>, dim3(1), dim3(TriCfg<NC>::THREADS), smem, M, k, level, lvl, gV, tri, scal);
}

void launch_seed_level(Launcher& L, const double* M, int k, int level, int32_t* lvl, float* gV, float* Zc, float* U,
                       float* Wk, float* tri, double* Xout, double* lam, double* scal, int32_t* stats,
                       int32_t* cid) {
  if (k <= 128)
    launch_pdl(L, seed_tri_col_kernel, dim3(1), dim3(kTC), 0, M, k, level, lvl, gV, tri, scal);
  else
    launch_tri<256>(L, M, k, level, lvl, gV, tri, scal);
  launch_pdl(L, seed_bisect_kernel, dim3((k + 3) / 4), dim3(128), 0, k, level, lvl, tri);
  const size_t sii = (size_t)2 * 33 * 256 * sizeof(float);
  cudaFuncSetAttribute(seed_ii_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sii);
  launch_pdl(L, seed_ii_kernel, dim3((k + kIIThreads - 1) / kIIThreads), dim3(kIIThreads), sii, k, level, lvl, tri, Zc);
  launch_pdl(L, seed_orth_kernel, dim3(1), dim3(kOrthThreads), 0, k, level, lvl, tri, Zc, U, Wk, stats, cid);
  const size_t sback = (size_t)((k * (k - 1)) / 2 + 4) * sizeof(float);
  cudaFuncSetAttribute(seed_back_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sback);
  launch_pdl(L, seed_back_kernel, dim3((k + kBackWarps - 1) / kBackWarps), dim3(kBackWarps * 32), sback, k, level, lvl, gV, Zc, tri, Xout, lam);
  L.count(5);
}

}  // namespace lspca
