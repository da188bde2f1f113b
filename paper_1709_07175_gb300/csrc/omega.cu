// K0: Omega on the device (Sec. I-A).  Dense materialisation (row-major n x k or
// transposed k x n) in FP64/FP32/BF16, and the very sparse kind as per-column
// signed index lists (CSC), generated in row order so every list is sorted.
#include "common.cuh"
#include "kernels.h"
#include "philox.cuh"

namespace lspca {

// One thread per (row i, word block b): one Philox call -> columns 4b..4b+3.
template <typename OutT>
__global__ void omega_dense_kernel(lspca_omega om, int64_t n, int k, OutT* out, int64_t ld, int transposed,
                                   int bf16_round) {
  const int nb = (k + 3) >> 2;
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= n * (int64_t)nb) return;
  const uint32_t i = (uint32_t)(idx / nb);
  const uint32_t b = (uint32_t)(idx % nb);
  float vals[4];
  if (om.kind == LSPCA_OMEGA_GAUSSIAN) {
    const uint4 w = omega_words(om.seed, i, b, kTagGaussian);
    vals[0] = gaussian_from_pair(w.x, w.y, false);
    vals[1] = gaussian_from_pair(w.x, w.y, true);
    vals[2] = gaussian_from_pair(w.z, w.w, false);
    vals[3] = gaussian_from_pair(w.z, w.w, true);
    if (bf16_round) {
#pragma unroll
      for (int q = 0; q < 4; ++q) vals[q] = __bfloat162float(__float2bfloat16_rn(vals[q]));
    }
  } else {
    const uint4 w = omega_words(om.seed, i, b, kTagSparse);
    const uint64_t t = sparse_threshold(om.p);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const uint64_t r = word_of(w, q);
      vals[q] = r < t ? -1.f : (r < 2 * t ? 1.f : 0.f);
    }
  }
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int j = 4 * (int)b + q;
    if (j >= k) break;
    const int64_t off = transposed ? (int64_t)j * ld + i : (int64_t)i * ld + j;
    out[off] = OutT(vals[q]);
  }
}

// Very sparse Omega -> CSC.  One warp per column c; lanes walk the rows in order
// and a ballot compacts the nonzeros, so each column's list is sorted by row.
// Entry encoding: e = s * (i + 1), s = +-1.
__global__ void omega_csc_count_kernel(lspca_omega om, int64_t n, int k, int32_t* counts) {
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (warp >= k) return;
  const int c = warp;
  int cnt = 0;
  for (int64_t i0 = 0; i0 < n; i0 += 32) {
    const int64_t i = i0 + lane;
    int v = 0;
    if (i < n) v = omega_sparse_entry(om.seed, om.p, (uint32_t)i, (uint32_t)c);
    cnt += __popc(__ballot_sync(0xffffffffu, v != 0));
  }
  if (lane == 0) counts[c] = cnt;
}

// Exclusive scan of k <= 4096 counts by one block.
__global__ void omega_csc_scan_kernel(const int32_t* counts, int k, int32_t* col_ptr) {
  __shared__ int32_t buf[4097];
  for (int c = threadIdx.x; c < k; c += blockDim.x) buf[c] = counts[c];
  __syncthreads();
  if (threadIdx.x == 0) {
    int32_t acc = 0;
    for (int c = 0; c < k; ++c) {
      const int32_t v = buf[c];
      buf[c] = acc;
      acc += v;
    }
    buf[k] = acc;
  }
  __syncthreads();
  for (int c = threadIdx.x; c <= k; c += blockDim.x) col_ptr[c] = buf[c];
}

__global__ void omega_csc_fill_kernel(lspca_omega om, int64_t n, int k, const int32_t* col_ptr, int32_t* entries) {
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (warp >= k) return;
  const int c = warp;
  int32_t pos = col_ptr[c];
  for (int64_t i0 = 0; i0 < n; i0 += 32) {
    const int64_t i = i0 + lane;
    int v = 0;
    if (i < n) v = omega_sparse_entry(om.seed, om.p, (uint32_t)i, (uint32_t)c);
    const unsigned bal = __ballot_sync(0xffffffffu, v != 0);
    if (v != 0) {
      const int before = __popc(bal & ((1u << lane) - 1u));
      entries[pos + before] = v * (int32_t)(i + 1);
    }
    pos += __popc(bal);
  }
}

void launch_omega_dense(Launcher& L, const lspca_omega& om, int64_t n, int k, int out_dt, void* out, int64_t ld,
                        bool transposed, bool bf16_round) {
  const int nb = (k + 3) / 4;
  const int64_t total = n * nb;
  const int threads = 256;
  const int blocks = (int)((total + threads - 1) / threads);
  switch (out_dt) {
    case LSPCA_F64:
      omega_dense_kernel<double><<<blocks, threads, 0, L.stream>>>(om, n, k, (double*)out, ld, transposed, bf16_round);
      break;
    case LSPCA_F32:
      omega_dense_kernel<float><<<blocks, threads, 0, L.stream>>>(om, n, k, (float*)out, ld, transposed, bf16_round);
      break;
    case LSPCA_BF16:
      omega_dense_kernel<__nv_bfloat16>
          <<<blocks, threads, 0, L.stream>>>(om, n, k, (__nv_bfloat16*)out, ld, transposed, bf16_round);
      break;
  }
  L.count(1);
}

void launch_omega_csc(Launcher& L, const lspca_omega& om, int64_t n, int k, int32_t* counts, int32_t* col_ptr,
                      int32_t* entries) {
  const int threads = 256;
  const int blocks = (k * 32 + threads - 1) / threads;
  omega_csc_count_kernel<<<blocks, threads, 0, L.stream>>>(om, n, k, counts);
  omega_csc_scan_kernel<<<1, 256, 0, L.stream>>>(counts, k, col_ptr);
  omega_csc_fill_kernel<<<blocks, threads, 0, L.stream>>>(om, n, k, col_ptr, entries);
  L.count(3);
}

}  // namespace lspca
