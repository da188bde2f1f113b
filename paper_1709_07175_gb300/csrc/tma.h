// Host-side construction of TMA tensor maps (driver entry point looked up once
// through the runtime, so the library does not link libcuda directly).
#pragma once

#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>

#include <mutex>

namespace lspca {

// Row-major 2-D tensor (rows x cols, row pitch ld_bytes) with a box of
// box_rows x box_cols elements and the 128-byte swizzle (box_cols * elem must
// be 128 bytes).  Out-of-range elements of a box are filled with zeros.
// Returns false when the driver entry point is missing or rejects the map
// (base not 16-byte aligned, pitch not a multiple of 16 bytes, ...).
inline bool make_tmap_2d_sw128(CUtensorMap* out, const void* base, CUtensorMapDataType dt, int elem_bytes,
                               uint64_t rows, uint64_t cols, uint64_t ld_bytes, uint32_t box_rows,
                               uint32_t box_cols) {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(f);
    cudaGetLastError();
  });
  if (!fn || box_cols * (uint32_t)elem_bytes != 128u) return false;
  const cuuint64_t dims[2] = {cols, rows};
  const cuuint64_t strides[1] = {ld_bytes};
  const cuuint32_t box[2] = {box_cols, box_rows};
  const cuuint32_t estr[2] = {1, 1};
  return fn(out, dt, 2, const_cast<void*>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
            CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) ==
         CUDA_SUCCESS;
}

}  // namespace lspca
