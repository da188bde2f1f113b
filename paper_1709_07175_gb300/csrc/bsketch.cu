// Pass S for FP8 E4M3 X with the very sparse Omega (Eq. 1, Alg. 2 step 1):
// U = X Omega as a gather over the nonzeros of X.
//
// The intended E4M3 input is binary features (Experiment 1 of the paper: a
// mostly-binary, sparse design matrix).  Omega has about k / p nonzeros per
// row, so row i of U is the sum, over the nonzero x_ij of row i, of x_ij times
// the few signed entries of row j of Omega: about nnz(x_i) k / p additions
// per row (Prop. 4: the sketch costs O(nnz(X) l)), far below the 4 n k
// multiply-adds of the dense product, while the n bytes of every row must be
// read anyway.  The kernel is therefore bound by reading X.
//
// Exactness.  Every E4M3 value is an integer multiple of 2^-9 of magnitude at
// most 448, so U is accumulated in int32 units of 2^-9 (shared-memory integer
// atomics: order-independent, bit-reproducible) and converted once; the
// result is exact whenever |U| < 2^15 (|U| 2^9 < 2^24), which holds by a wide
// margin for binary features.
//
// Structure.  Omega's nonzeros are first described per row, built on the
// device from the same Philox stream as every other Omega form: one 16-byte
// word per row j holds the count (4 bits), up to 12 signs and 12 column bytes;
// rows with more nonzeros (rare at p >= 16) are marked and also listed in a
// CSR (rp / ent).  Each warp of the sketch owns one row of X at a time: every
// lane loads 16-byte words of the row (512 bytes per warp instruction), finds
// the nonzero bytes of each 32-bit word with three integer operations, and for
// each one adds its scaled value, once per nonzero of Omega's row, into the
// row's int32 accumulator in shared memory.
#include "common.cuh"
#include "kernels.h"
#include "philox.cuh"

namespace lspca {
namespace {

constexpr int kBsWarps = 8;
constexpr int kBsWords = 8;   // 16-byte words per lane per pass (4 KB of a row per warp)
constexpr int kBsInline = 12; // Omega nonzeros held in a row's descriptor word

// Omega rows: count the nonzeros of each row j (one thread per row).
__global__ void omega_rows_count_kernel(lspca_omega om, int64_t n, int k, int32_t* cnt) {
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  const uint64_t t = sparse_threshold(om.p);
  int c = 0;
  for (int b = 0; b * 4 < k; ++b) {
    const uint4 w = omega_words(om.seed, (uint32_t)j, (uint32_t)b, kTagSparse);
#pragma unroll
    for (int q = 0; q < 4; ++q)
      if (4 * b + q < k) c += (uint64_t)word_of(w, q) < 2 * t;
  }
  cnt[j] = c;
}

// Exclusive prefix of the n row counts (one block; rp[n] = nnz).
__global__ void __launch_bounds__(1024) omega_rows_scan_kernel(const int32_t* cnt, int64_t n, int32_t* rp) {
  __shared__ int32_t part[1024];
  const int tid = threadIdx.x;
  const int64_t per = (n + 1023) / 1024;
  const int64_t a = tid * per, b = min(n, a + per);
  int32_t s = 0;
  for (int64_t j = a; j < b; ++j) s += cnt[j];
  part[tid] = s;
  __syncthreads();
  if (tid == 0) {
    int32_t acc = 0;
    for (int i = 0; i < 1024; ++i) {
      const int32_t v = part[i];
      part[i] = acc;
      acc += v;
    }
    rp[n] = acc;
  }
  __syncthreads();
  int32_t acc = part[tid];
  for (int64_t j = a; j < b; ++j) {
    rp[j] = acc;
    acc += cnt[j];
  }
}

// Omega rows: the CSR list of row j in column order (e = s (l + 1)) and the
// row's descriptor word: x bits 0-3 count (15: more than kBsInline, use the
// list), bits 4-15 signs (1 = -1) of the first 12; bytes 2-3 of x and the
// bytes of y, z, w their columns.
__global__ void omega_rows_fill_kernel(lspca_omega om, int64_t n, int k, const int32_t* rp, int16_t* ent,
                                       uint4* desc) {
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  const uint64_t t = sparse_threshold(om.p);
  int32_t pos = rp[j];
  uint32_t d[4] = {0u, 0u, 0u, 0u};
  int c = 0;
  for (int b = 0; b * 4 < k; ++b) {
    const uint4 w = omega_words(om.seed, (uint32_t)j, (uint32_t)b, kTagSparse);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int l = 4 * b + q;
      const uint64_t r = word_of(w, q);
      if (l < k && r < 2 * t) {
        const bool neg = r < t;
        ent[pos++] = (int16_t)(neg ? -(l + 1) : (l + 1));
        if (c < kBsInline) {
          if (neg) d[0] |= 1u << (4 + c);
          const int byte = c + 2;  // column bytes start at byte 2 of x
          d[byte >> 2] |= (uint32_t)l << (8 * (byte & 3));
        }
        ++c;
      }
    }
  }
  d[0] |= (uint32_t)(c > kBsInline ? 15 : c);
  desc[j] = make_uint4(d[0], d[1], d[2], d[3]);
}

// E4M3 byte -> value in units of 2^-9 (exact), with NaN flagged.
__device__ __forceinline__ int e4m3_units(uint32_t b, bool& nan) {
  const uint32_t mag = b & 0x7Fu;
  if (mag == 0x7Fu) nan = true;
  const uint32_t e = mag >> 3, mt = mag & 7u;
  const int v = e ? (int)((8u + mt) << (e - 1)) : (int)mt;
  return (b & 0x80u) ? -v : v;
}

// Add v times row j of Omega into the accumulator a.
__device__ __forceinline__ void add_omega_row(int32_t* a, int v, uint4 d, int64_t j,
                                              const int32_t* __restrict__ rp, const int16_t* __restrict__ ent) {
  const int cnt = d.x & 15u;
  if (cnt == 15) {  // more nonzeros than the descriptor holds: the list
    const int32_t b0 = __ldg(rp + j), b1 = __ldg(rp + j + 1);
    for (int32_t t = b0; t < b1; ++t) {
      const int code = __ldg(ent + t);
      atomicAdd(&a[(code < 0 ? -code : code) - 1], code < 0 ? -v : v);
    }
    return;
  }
  const uint32_t words[4] = {d.x, d.y, d.z, d.w};
#pragma unroll
  for (int e = 0; e < kBsInline; ++e) {
    if (e >= cnt) break;
    const int byte = e + 2;
    const int col = (words[byte >> 2] >> (8 * (byte & 3))) & 0xFF;
    atomicAdd(&a[col], ((d.x >> (4 + e)) & 1u) ? -v : v);
  }
}

__global__ void __launch_bounds__(kBsWarps * 32) bsketch_kernel(const uint8_t* __restrict__ X, int64_t ldx,
                                                               int64_t m, int64_t n, int k,
                                                               const uint4* __restrict__ desc,
                                                               const int32_t* __restrict__ rp,
                                                               const int16_t* __restrict__ ent,
                                                               float* __restrict__ U, float* umax, int* status) {
  __shared__ int32_t acc[kBsWarps][256];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  int32_t* a = acc[w];
  for (int l = lane; l < 256; l += 32) a[l] = 0;
  __syncwarp();
  bool nan = false;
  float mx = 0.f;
  const int64_t nwords = (n + 15) / 16;  // 16-byte words of a row
  const int64_t gw = (int64_t)blockIdx.x * kBsWarps + w, nw = (int64_t)gridDim.x * kBsWarps;
  for (int64_t i = gw; i < m; i += nw) {
    const uint8_t* row = X + i * ldx;
    for (int64_t w0 = 0; w0 < nwords; w0 += 32 * kBsWords) {
      uint4 wv[kBsWords];
#pragma unroll
      for (int u = 0; u < kBsWords; ++u) {
        const int64_t wi = w0 + u * 32 + lane;
        wv[u] = wi < nwords ? __ldcs(reinterpret_cast<const uint4*>(row) + wi) : make_uint4(0u, 0u, 0u, 0u);
      }
#pragma unroll
      for (int u = 0; u < kBsWords; ++u) {
        const int64_t col0 = (w0 + u * 32 + lane) * 16;  // column of the word's first byte
        const uint32_t q4[4] = {wv[u].x, wv[u].y, wv[u].z, wv[u].w};
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          // bit 7 of each byte: magnitude nonzero (the sign of -0 ignored)
          uint32_t nz = ((q4[q] & 0x7F7F7F7Fu) + 0x7F7F7F7Fu) & 0x80808080u;
          const int64_t cq = col0 + 4 * q;
          if (cq + 4 > n && nz) {  // the row's last word: bytes past n are padding
            const int valid = (int)(n - cq);
            nz &= valid <= 0 ? 0u : (valid >= 4 ? 0xFFFFFFFFu : ((1u << (8 * valid)) - 1u));
          }
          while (nz) {
            const int bit = __ffs(nz) - 1;
            nz &= nz - 1;
            const int64_t j = cq + (bit >> 3);
            const int v = e4m3_units((q4[q] >> (bit - 7)) & 0xFFu, nan);
            add_omega_row(a, v, __ldg(desc + j), j, rp, ent);
          }
        }
      }
    }
    __syncwarp();
    // U row i (units of 2^-9 -> FP32), and a cleared accumulator for the next row
    float* ur = U + i * (int64_t)k;
    for (int l = lane; l < k; l += 32) {
      const float v = (float)a[l] * 0x1p-9f;
      ur[l] = v;
      mx = fmaxf(mx, fabsf(v));
      a[l] = 0;
    }
    __syncwarp();
  }
  mx = warp_max(mx);
  if (lane == 0 && mx > 0.f) atomic_max_nonneg(umax, mx);
  if (__any_sync(0xffffffffu, nan) && lane == 0) atomicOr(status, ST_NONFINITE);
}

size_t rows_bytes(int64_t n) { return ((size_t)(n + 1) * 4 + 255) / 256 * 256; }

}  // namespace

size_t bsketch_ws_bytes(int64_t n, int k) {
  return 2 * rows_bytes(n) + ((size_t)n * k * 2 + 255) / 256 * 256 + ((size_t)n * 16 + 255) / 256 * 256;
}

void launch_bsketch(Launcher& L, const void* X, int64_t m, int64_t n, int64_t ldx, int k, const lspca_omega& om,
                    void* ws, float* U, float* umax, int* status) {
  char* p = (char*)ws;
  int32_t* rp = (int32_t*)p;
  p += rows_bytes(n);
  int32_t* cnt = (int32_t*)p;
  p += rows_bytes(n);
  uint4* desc = (uint4*)p;
  p += ((size_t)n * 16 + 255) / 256 * 256;
  int16_t* ent = (int16_t*)p;
  const int blocks = (int)((n + 255) / 256);
  omega_rows_count_kernel<<<blocks, 256, 0, L.stream>>>(om, n, k, cnt);
  omega_rows_scan_kernel<<<1, 1024, 0, L.stream>>>(cnt, n, rp);
  omega_rows_fill_kernel<<<blocks, 256, 0, L.stream>>>(om, n, k, rp, ent, desc);
  // enough resident warps to keep X's loads in flight: 6 CTAs of 8 warps per SM
  int64_t grid = (int64_t)L.num_sms * 6;
  const int64_t need = (m + kBsWarps - 1) / kBsWarps;
  if (grid > need) grid = need;
  if (grid < 1) grid = 1;
  bsketch_kernel<<<(unsigned)grid, kBsWarps * 32, 0, L.stream>>>((const uint8_t*)X, ldx, m, n, k, desc, rp, ent, U,
                                                                 umax, status);
  L.count(4);
}

}  // namespace lspca
