// Shared device/host helpers of liblspca (types, loads, status word, launch bookkeeping).
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_fp8.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/lspca.h"

namespace lspca {

// Device status bits (set with atomicOr by the kernels, read by the host after sync).
enum : int {
  ST_NONFINITE = 1,   // NaN or Inf found in X
  ST_TIMEOUT = 2,     // a bounded wait gave up
  ST_NUMERIC = 4,     // eigensolver did not converge within its sweep limit
  ST_BADINDEX = 8,    // a sparse X's column index outside [0, n)
};

// Programmatic dependent launch.  A kernel launched with launch_pdl is set up
// by the GPU while its predecessor in the stream still runs and starts as the
// predecessor ends; pdl_wait blocks until the predecessor has completed and
// its writes are visible.  Every such kernel calls pdl_wait first and
// unconditionally (also on paths that return early), so completion stays
// ordered along the chain: kernel i ends only after kernel i - 1 ended.
// (Letting successors be scheduled early with griddepcontrol.launch_dependents
// was slower: their waiting CTAs took SMs from the running kernels.)  A no-op
// for a kernel launched without PDL.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

// Element access: every X element type decodes exactly to float (F32/BF16/E4M3)
// or double (F64).
template <int DT> struct XType;
template <> struct XType<LSPCA_F64> {
  using T = double;
  using Acc = double;
  __device__ __forceinline__ static double to_acc(T v) { return v; }
};
template <> struct XType<LSPCA_F32> {
  using T = float;
  using Acc = float;
  __device__ __forceinline__ static float to_acc(T v) { return v; }
};
template <> struct XType<LSPCA_BF16> {
  using T = __nv_bfloat16;
  using Acc = float;
  __device__ __forceinline__ static float to_acc(T v) { return __bfloat162float(v); }
};
template <> struct XType<LSPCA_E4M3> {
  using T = __nv_fp8_e4m3;
  using Acc = float;
  __device__ __forceinline__ static float to_acc(T v) { return float(v); }
};

inline size_t dtype_size(int dt) {
  switch (dt) {
    case LSPCA_F64: return 8;
    case LSPCA_F32: return 4;
    case LSPCA_BF16: return 2;
    case LSPCA_E4M3: return 1;
    default: return 0;
  }
}

__device__ __forceinline__ bool finite_acc(float v) { return isfinite(v); }
__device__ __forceinline__ bool finite_acc(double v) { return isfinite(v); }

__device__ __forceinline__ float abs_acc(float v) { return fabsf(v); }
__device__ __forceinline__ double abs_acc(double v) { return fabs(v); }

// Max of non-negative floats through their bit patterns (order-independent).
__device__ __forceinline__ void atomic_max_nonneg(float* addr, float v) {
  atomicMax(reinterpret_cast<unsigned int*>(addr), __float_as_uint(v));
}

__device__ __forceinline__ float warp_max(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ __forceinline__ float warp_sumf(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

inline int ceil_div(int64_t a, int64_t b) { return (int)((a + b - 1) / b); }

}  // namespace lspca
