// Device Philox4x32-10 and the Omega entry generators.
//
// Philox4x32-10 is written from its published definition (Salmon, Moraes,
// Dror, Shaw, "Parallel random numbers: as easy as 1, 2, 3", SC'11): ten
// rounds of two 32x32->64 multiplications with multipliers 0xD2511F53 and
// 0xCD9E8D57, the high halves xored with the other two words and the round
// key, and a Weyl key schedule with increments 0x9E3779B9 / 0xBB67AE85.
//
// Omega (Sec. I-A of the paper): Gaussian N(0, 1) entries, or very sparse
// entries in {-1, 0, +1} with probabilities {1/2p, 1 - 1/p, 1/2p}.  Entry
// (i, j) of the n x k matrix draws from counter (i, j / 4, tag, 0) and key
// (seed mod 2^32, seed / 2^32); word j % 4 feeds column j.
#pragma once

#include <stdint.h>

namespace lspca {

constexpr uint32_t kTagGaussian = 0;
constexpr uint32_t kTagSparse = 1;

__host__ __device__ __forceinline__ uint32_t mulhi32(uint32_t a, uint32_t b) {
#ifdef __CUDA_ARCH__
  return __umulhi(a, b);
#else
  return (uint32_t)(((uint64_t)a * (uint64_t)b) >> 32);
#endif
}

__host__ __device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r) {
      k0 += 0x9E3779B9u;
      k1 += 0xBB67AE85u;
    }
    const uint32_t hi0 = mulhi32(0xD2511F53u, c.x), lo0 = 0xD2511F53u * c.x;
    const uint32_t hi1 = mulhi32(0xCD9E8D57u, c.z), lo1 = 0xCD9E8D57u * c.z;
    c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
  }
  return c;
}

__device__ __forceinline__ uint4 omega_words(uint64_t seed, uint32_t i, uint32_t block, uint32_t tag) {
  return philox4x32_10(make_uint4(i, block, tag, 0u), (uint32_t)seed, (uint32_t)(seed >> 32));
}

__device__ __forceinline__ uint32_t word_of(uint4 w, int q) {
  return q == 0 ? w.x : q == 1 ? w.y : q == 2 ? w.z : w.w;
}

// Box-Muller on one word pair; returns the cos (even column) or sin (odd) value
// rounded to FP32.  u = (w + 1/2) 2^-32 lies in (0, 1).
__device__ __forceinline__ float gaussian_from_pair(uint32_t wa, uint32_t wb, bool sine) {
  const double ua = ((double)wa + 0.5) * 0x1p-32;
  const double ub = ((double)wb + 0.5) * 0x1p-32;
  const double rad = sqrt(-2.0 * log(ua));
  double s, c;
  sincospi(2.0 * ub, &s, &c);
  return __double2float_rn(rad * (sine ? s : c));
}

// Omega_ij, Gaussian kind, as FP32.
__device__ __forceinline__ float omega_gaussian_entry(uint64_t seed, uint32_t i, uint32_t j) {
  const uint4 w = omega_words(seed, i, j >> 2, kTagGaussian);
  const int q = j & 3;
  const uint32_t wa = (q < 2) ? w.x : w.z;
  const uint32_t wb = (q < 2) ? w.y : w.w;
  return gaussian_from_pair(wa, wb, (q & 1) != 0);
}

__host__ __device__ __forceinline__ uint32_t sparse_threshold(uint32_t p) {
  return (uint32_t)((1ull << 32) / (2ull * (uint64_t)p));
}

// Omega_ij, very sparse kind: -1, 0 or +1.
__device__ __forceinline__ int omega_sparse_entry(uint64_t seed, uint32_t p, uint32_t i, uint32_t j) {
  const uint4 w = omega_words(seed, i, j >> 2, kTagSparse);
  const uint32_t r = word_of(w, j & 3);
  const uint64_t t = sparse_threshold(p);
  if ((uint64_t)r < t) return -1;
  if ((uint64_t)r < 2ull * t) return 1;
  return 0;
}

}  // namespace lspca
