// Sparse X in CSR form (rows = samples): the sketch U = X Omega, pass F
// (F = U^T X, Algorithm 2 step 2) and the reduction map Y = X V for a data
// matrix given by its nonzeros, the format of the paper's experiments (sparse
// slices, Sec. IV).  The work is proportional to nnz(X) (Prop. 4's nnz(X) l
// terms), so these kernels are plain SIMT gathers with compensated FP32 dot
// products (exact products, Neumaier sums: a few ulps, at FP32 rates):
//
//   rows:   Y[i, :] = sum over the nonzeros (j, x) of row i of x D[j, :]
//           (D = Omega for the sketch, V for the reduction map), one warp per
//           row, lanes over the k columns;
//   pass F: F[:, j] = sum over the nonzeros (i, x) of column j of x U[i, :]
//           over a CSC copy of X whose entries are in row order: one warp per
//           segment of up to 128 entries of a column, then one warp per column
//           adds its segments' partials in order, so every sum has a fixed
//           order (no atomics on F) and a heavy column is spread over warps.
//
// The CSC copy is a stable counting sort by column: per block of S rows the
// column counts (hist), their prefix over the blocks and columns (offsets),
// then one warp per row block places its nonzeros row by row (positions
// taken with atomicAdd on the block's own offsets: distinct columns of one
// row never share a counter, so the order within a column is the row order;
// duplicate (i, j) entries of one row, which CSR allows, land in an
// unspecified order).  Column indices outside [0, n) and row offsets that are
// not a nondecreasing sequence from 0 to nnz set ST_BADINDEX (such entries are
// skipped, offsets clamped to [0, nnz]); NaN / Inf values set ST_NONFINITE.
#include "common.cuh"
#include "kernels.h"

namespace lspca {

namespace {

// Compensated FP32 dot product: the product x d is taken exactly as y + e
// (y rounded, e = fma(x, d, -y) its error) and the sum by Neumaier's method,
// s + c then carries the sum to a few ulps whatever the number of terms, at
// FP32 rates (GB300 runs FP64 FMAs at 1/64 of the FP32 rate).  The rounded
// product is formed on its own (no contraction into the sum), as the
// compensation assumes.
__device__ __forceinline__ void nsum_add(float& s, float& c, float x, float d) {
  const float y = __fmul_rn(x, d);
  const float e = fmaf(x, d, -y);
  const float t = __fadd_rn(s, y);
  const float r = fabsf(s) >= fabsf(y) ? __fadd_rn(__fsub_rn(s, t), y) : __fadd_rn(__fsub_rn(y, t), s);
  c = __fadd_rn(c, __fadd_rn(r, e));
  s = t;
}

// A row offset clamped to [0, nnz]: inconsistent offsets (flagged by the row
// kernel) never take a kernel outside the arrays.
__device__ __forceinline__ int64_t clamp_nnz(int64_t p, int64_t nnz) { return p < 0 ? 0 : (p > nnz ? nnz : p); }

// Y[i, :] = sum_p val[p] D[col[p], :]; compensated FP32 sums, FP32 output.
__global__ void __launch_bounds__(256) csr_rows_kernel(const int64_t* __restrict__ row_ptr,
                                                       const int32_t* __restrict__ col,
                                                       const float* __restrict__ val, int64_t m, int64_t n,
                                                       int64_t nnz, const float* __restrict__ D, int k,
                                                       float* __restrict__ Y, int* status) {
  const int lane = threadIdx.x & 31;
  const int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (i >= m) return;
  float acc[8] = {0, 0, 0, 0, 0, 0, 0, 0}, cmp[8] = {0, 0, 0, 0, 0, 0, 0, 0};  // columns lane + 32 t, k <= 256
  const int64_t a = row_ptr[i], e = row_ptr[i + 1];
  int bad = (e < a || a < 0 || e > nnz || (i == 0 && a != 0) || (i == m - 1 && e != nnz)) ? ST_BADINDEX : 0;
  const int64_t p0 = clamp_nnz(a, nnz), p1 = clamp_nnz(e, nnz);
  for (int64_t p = p0; p < p1; ++p) {
    const int32_t j = col[p];
    const float x = val[p];
    if (!isfinite(x)) bad |= ST_NONFINITE;
    if (j < 0 || j >= n) {
      bad |= ST_BADINDEX;
      continue;
    }
    const float* d = D + (int64_t)j * k;
#pragma unroll
    for (int t = 0; t < 8; ++t) {
      const int c = lane + 32 * t;
      if (c < k) nsum_add(acc[t], cmp[t], x, d[c]);
    }
  }
#pragma unroll
  for (int t = 0; t < 8; ++t) {
    const int c = lane + 32 * t;
    if (c < k) Y[i * k + c] = __fadd_rn(acc[t], cmp[t]);
  }
  if (bad && lane == 0) atomicOr(status, bad);
}

// Column counts of the rows of block b: hist[b * n + j] (int64).
__global__ void csr_hist_kernel(const int64_t* __restrict__ row_ptr, const int32_t* __restrict__ col, int64_t m,
                                int64_t n, int64_t nnz, int64_t rows_per_block, unsigned long long* hist) {
  const int64_t b = blockIdx.x;
  const int64_t r0 = b * rows_per_block, r1 = min(m, r0 + rows_per_block);
  for (int64_t i = r0; i < r1; ++i) {  // the same clamped ranges as the row kernel
    const int64_t p0 = clamp_nnz(row_ptr[i], nnz), p1 = clamp_nnz(row_ptr[i + 1], nnz);
    for (int64_t p = p0 + threadIdx.x; p < p1; p += blockDim.x) {
      const int32_t j = col[p];
      if (j >= 0 && j < n) atomicAdd(&hist[b * n + j], 1ull);
    }
  }
}

// Per column j: total count over the blocks (into cnt[j]), sequentially over b.
__global__ void csc_count_kernel(const unsigned long long* __restrict__ hist, int64_t nblocks, int64_t n,
                                 int64_t* cnt) {
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  unsigned long long s = 0;
  int64_t b = 0;
  for (; b + 8 <= nblocks; b += 8) {  // eight loads in flight, summed in order
    unsigned long long c[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) c[u] = hist[(b + u) * n + j];
#pragma unroll
    for (int u = 0; u < 8; ++u) s += c[u];
  }
  for (; b < nblocks; ++b) s += hist[b * n + j];
  cnt[j] = (int64_t)s;
}

// Exclusive scan of cnt[0 .. n) into col_ptr[0 .. n] by one block: each thread
// sums a contiguous range, the block scans those sums, each thread rewrites
// its range.
__global__ void __launch_bounds__(1024) scan_kernel(const int64_t* __restrict__ cnt, int64_t n, int64_t* col_ptr) {
  __shared__ int64_t part[1024];
  const int t = threadIdx.x, T = blockDim.x;
  const int64_t per = (n + T - 1) / T;
  const int64_t a = min(n, per * t), e = min(n, a + per);
  int64_t s = 0;
  for (int64_t j = a; j < e; ++j) s += cnt[j];
  part[t] = s;
  __syncthreads();
  if (t == 0) {
    int64_t run = 0;
    for (int i = 0; i < T; ++i) {
      const int64_t v = part[i];
      part[i] = run;
      run += v;
    }
    col_ptr[n] = run;
  }
  __syncthreads();
  int64_t run = part[t];
  for (int64_t j = a; j < e; ++j) {
    col_ptr[j] = run;
    run += cnt[j];
  }
}

// hist[b * n + j] <- the CSC position of block b's first entry in column j:
// col_ptr[j] + the counts of the earlier blocks.
__global__ void csc_offsets_kernel(unsigned long long* hist, int64_t nblocks, int64_t n,
                                   const int64_t* __restrict__ col_ptr) {
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  unsigned long long run = (unsigned long long)col_ptr[j];
  int64_t b = 0;
  for (; b + 8 <= nblocks; b += 8) {  // eight loads in flight, the prefix in order
    unsigned long long c[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) c[u] = hist[(b + u) * n + j];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      hist[(b + u) * n + j] = run;
      run += c[u];
    }
  }
  for (; b < nblocks; ++b) {
    const unsigned long long c = hist[b * n + j];
    hist[b * n + j] = run;
    run += c;
  }
}

// One warp per row block: the block's rows in order, each row's nonzeros by
// the lanes; crow / cval receive the row index and the value at the CSC position.
__global__ void csc_fill_kernel(const int64_t* __restrict__ row_ptr, const int32_t* __restrict__ col,
                                const float* __restrict__ val, int64_t m, int64_t n, int64_t nnz,
                                int64_t rows_per_block, int64_t nblocks, unsigned long long* offs,
                                int32_t* __restrict__ crow, float* __restrict__ cval) {
  const int lane = threadIdx.x & 31;
  const int64_t b = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (b >= nblocks) return;
  const int64_t r0 = b * rows_per_block, r1 = min(m, r0 + rows_per_block);
  unsigned long long* o = offs + b * n;
  for (int64_t i = r0; i < r1; ++i) {
    const int64_t p0 = clamp_nnz(row_ptr[i], nnz), p1 = clamp_nnz(row_ptr[i + 1], nnz);
    for (int64_t p = p0 + lane; p < p1; p += 32) {
      const int32_t j = col[p];
      if (j < 0 || j >= n) continue;
      const unsigned long long pos = atomicAdd(&o[j], 1ull);
      if (pos < (unsigned long long)nnz) {  // only inconsistent offsets count more than nnz entries
        crow[pos] = (int32_t)i;
        cval[pos] = val[p];
      }
    }
    __syncwarp();  // the next row's positions come after this row's
  }
}

constexpr int kSeg = 128;  // CSC entries per pass-F segment

// Segments per column: ceil(entries / kSeg).
__global__ void seg_count_kernel(const int64_t* __restrict__ col_ptr, int64_t n, int64_t* segc) {
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j < n) segc[j] = (col_ptr[j + 1] - col_ptr[j] + kSeg - 1) / kSeg;
}

// One warp per segment s of column j (seg_ptr[j] <= s < seg_ptr[j + 1]):
// P[s, :] = sum over the segment's entries (row order) of x U[i, :]
// (compensated FP32 sum, written as the FP64 value s + c).
__global__ void __launch_bounds__(256) passf_seg_kernel(const int64_t* __restrict__ col_ptr,
                                                        const int32_t* __restrict__ crow,
                                                        const float* __restrict__ cval, int64_t n, int64_t nnz,
                                                        const int64_t* __restrict__ seg_ptr,
                                                        const float* __restrict__ U, int k, double* __restrict__ P) {
  const int lane = threadIdx.x & 31;
  const int64_t s = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (s >= seg_ptr[n]) return;
  int64_t lo = 0, hi = n;  // the largest j with seg_ptr[j] <= s
  while (hi - lo > 1) {
    const int64_t mid = (lo + hi) >> 1;
    if (seg_ptr[mid] <= s) lo = mid;
    else hi = mid;
  }
  const int64_t j = lo;
  const int64_t p0 = col_ptr[j] + (s - seg_ptr[j]) * kSeg;
  const int64_t p1 = min(min(col_ptr[j + 1], p0 + kSeg), nnz);  // nnz: see csc_fill_kernel
  float acc[8] = {0, 0, 0, 0, 0, 0, 0, 0}, cmp[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  int64_t p = p0;
  for (; p + 4 <= p1; p += 4) {  // four entries' loads in flight at once
    int64_t i[4];
    float x[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      i[u] = crow[p + u];
      x[u] = cval[p + u];
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const float* r = U + i[u] * k;
#pragma unroll
      for (int t = 0; t < 8; ++t) {
        const int c = lane + 32 * t;
        if (c < k) nsum_add(acc[t], cmp[t], x[u], r[c]);
      }
    }
  }
  for (; p < p1; ++p) {
    const float* r = U + (int64_t)crow[p] * k;
    const float x = cval[p];
#pragma unroll
    for (int t = 0; t < 8; ++t) {
      const int c = lane + 32 * t;
      if (c < k) nsum_add(acc[t], cmp[t], x, r[c]);
    }
  }
#pragma unroll
  for (int t = 0; t < 8; ++t) {
    const int c = lane + 32 * t;
    if (c < k) P[s * k + c] = (double)acc[t] + (double)cmp[t];
  }
}

// One warp per column j: F[c, j] = sum of its segments' partials in order;
// F is k x n FP64 row-major (a column without entries gets zeros).
__global__ void __launch_bounds__(256) passf_reduce_kernel(const int64_t* __restrict__ seg_ptr, int64_t n,
                                                           const double* __restrict__ P, int k,
                                                           double* __restrict__ F) {
  const int lane = threadIdx.x & 31;
  const int64_t j = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (j >= n) return;
  double acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  for (int64_t s = seg_ptr[j]; s < seg_ptr[j + 1]; ++s) {
#pragma unroll
    for (int t = 0; t < 8; ++t) {
      const int c = lane + 32 * t;
      if (c < k) acc[t] += P[s * k + c];
    }
  }
#pragma unroll
  for (int t = 0; t < 8; ++t) {
    const int c = lane + 32 * t;
    if (c < k) F[(int64_t)c * n + j] = acc[t];
  }
}

}  // namespace

void launch_csr_rows(Launcher& L, const int64_t* row_ptr, const int32_t* col, const float* val, int64_t m, int64_t n,
                     int64_t nnz, const float* D, int k, float* Y, int* status) {
  if (m <= 0) return;
  const int64_t warps = m;
  const int64_t blocks = (warps * 32 + 255) / 256;
  csr_rows_kernel<<<(unsigned)blocks, 256, 0, L.stream>>>(row_ptr, col, val, m, n, nnz, D, k, Y, status);
  L.count(1);
}

int64_t csr_rows_per_block(int64_t m, int64_t n) {
  // keep the per-block column counters (8 bytes each) near 256 MB at most
  int64_t s = 256;
  while (s < m && (m + s - 1) / s * n > ((int64_t)32 << 20)) s *= 2;
  return s;
}

static int64_t max_segments(int64_t n, int64_t nnz) { return n + nnz / kSeg + 1; }

size_t csc_ws_bytes(int64_t m, int64_t n, int64_t nnz, int k) {
  const int64_t s = csr_rows_per_block(m, n);
  const int64_t nb = (m + s - 1) / s;
  return (size_t)nb * n * 8 + (size_t)n * 8 + (size_t)(n + 1) * 8 + (size_t)nnz * 8 + (size_t)n * 8 +
         (size_t)(n + 1) * 8 + (size_t)max_segments(n, nnz) * k * 8 + 10 * 256;
}

void launch_csr_to_csc(Launcher& L, const int64_t* row_ptr, const int32_t* col, const float* val, int64_t m,
                       int64_t n, int64_t nnz, int k, void* ws, CscView* out) {
  const int64_t s = csr_rows_per_block(m, n);
  const int64_t nb = (m + s - 1) / s;
  char* p = (char*)ws;
  auto take = [&](size_t bytes) {
    char* r = p;
    p += (bytes + 255) & ~(size_t)255;
    return r;
  };
  unsigned long long* hist = (unsigned long long*)take((size_t)nb * n * 8);
  int64_t* cnt = (int64_t*)take((size_t)n * 8);
  int64_t* col_ptr = (int64_t*)take((size_t)(n + 1) * 8);
  int32_t* crow = (int32_t*)take((size_t)nnz * 4);
  float* cval = (float*)take((size_t)nnz * 4);
  out->segc = (int64_t*)take((size_t)n * 8);
  out->seg_ptr = (int64_t*)take((size_t)(n + 1) * 8);
  out->part = (double*)take((size_t)max_segments(n, nnz) * k * 8);
  out->max_segments = max_segments(n, nnz);
  cudaMemsetAsync(hist, 0, (size_t)nb * n * 8, L.stream);
  csr_hist_kernel<<<(unsigned)nb, 256, 0, L.stream>>>(row_ptr, col, m, n, nnz, s, hist);
  const unsigned cb = (unsigned)((n + 255) / 256);
  csc_count_kernel<<<cb, 256, 0, L.stream>>>(hist, nb, n, cnt);
  scan_kernel<<<1, 1024, 0, L.stream>>>(cnt, n, col_ptr);
  csc_offsets_kernel<<<cb, 256, 0, L.stream>>>(hist, nb, n, col_ptr);
  csc_fill_kernel<<<(unsigned)((nb * 32 + 255) / 256), 256, 0, L.stream>>>(row_ptr, col, val, m, n, nnz, s, nb,
                                                                            hist, crow, cval);
  L.count(5);
  out->col_ptr = col_ptr;
  out->crow = crow;
  out->cval = cval;
}

void launch_csc_passf(Launcher& L, const CscView& c, int64_t n, int64_t nnz, const float* U, int k, double* F) {
  if (n <= 0) return;
  const unsigned cb = (unsigned)((n + 255) / 256);
  seg_count_kernel<<<cb, 256, 0, L.stream>>>(c.col_ptr, n, c.segc);
  scan_kernel<<<1, 1024, 0, L.stream>>>(c.segc, n, c.seg_ptr);
  passf_seg_kernel<<<(unsigned)((c.max_segments * 32 + 255) / 256), 256, 0, L.stream>>>(
      c.col_ptr, c.crow, c.cval, n, nnz, c.seg_ptr, U, k, c.part);
  passf_reduce_kernel<<<(unsigned)((n * 32 + 255) / 256), 256, 0, L.stream>>>(c.seg_ptr, n, c.part, k, F);
  L.count(4);
}

}  // namespace lspca
