// Tensor-core (tcgen05 / TMEM / TMA) passes of liblspca, sm_103a.
#pragma once

#include <stddef.h>
#include <stdint.h>

#include "kernels.h"

namespace lspca {

// True when the current device runs the tcgen05 kernels (compute capability 10.3).
bool tc_available();

// Pass F on tensor cores: F = U^T X and optionally G = U^T U.
struct TcChainWs {
  size_t bytes = 0;
  double* Fpart = nullptr;  // chunks x k x n FP32 partials
  double* Gpart = nullptr;  // gchunks x k x k FP32 partials
  int chunks = 1;
  int64_t rows_per_chunk = 0;
  int gchunks = 0;
  int64_t grows_per_chunk = 0;
  int64_t ku = 0;           // pitch (16-bit elements) of the split copies of U
  void* uhi = nullptr;      // m x ku: hi / lo 16-bit pairs of U (TMA-fed A operand)
  void* ulo = nullptr;
  void* ghi = nullptr;      // FP16 pairs of U for the Gram when X is BF16 / E4M3
  void* glo = nullptr;
};
// TMA-fed pass F (chain.cu): U is split once into 16-bit pairs in the workspace.
void plan_tc_chain(char* base, TcChainWs& w, int xt, int64_t m, int64_t n, int k, bool want_g, int num_sms);
// absmax[0] = max|X|, absmax[1] = max|U| on the device (FP32 / Gram scales).
// Returns false when a tensor map cannot be built or the kernel cannot be configured.
// gate (nullable): F's kernels do nothing unless *gate != 0 (the Gram always runs).
bool tc_chain_main(Launcher& L, const void* X, int xt, int64_t m, int64_t n, int64_t ldx, const float* U, int k,
                   TcChainWs& w, const float* absmax, int* status, bool want_g, const int* gate = nullptr);
// Pass F with U split inside the kernel (tc.cu): its workspace is the partials
// only, which a fixed-size scratch array can hold for any m.
void plan_tc_chain_inline(char* base, TcChainWs& w, int xt, int64_t m, int64_t n, int k, bool want_g, int num_sms);
void tc_chain_inline_main(Launcher& L, const void* X, int xt, int64_t m, int64_t n, int64_t ldx, const float* U,
                          int k, TcChainWs& w, const float* absmax, int* status, bool want_g);
// F (k x n FP64) = sum of the chunk partials, or F += that sum with accumulate (Algorithm 4's F += U_s^T X_s).
void tc_chain_reduce(Launcher& L, int64_t n, int k, TcChainWs& w, double* F, double* G, bool accumulate = false,
                     const int* gate = nullptr);

// Y = X V on tensor cores (FP32, BF16 or E4M3 X; V and Y FP32, k <= 256).  With V = a
// dense Omega the same kernel computes the sketch U = X Omega (pass S).
struct TcProjectWs {
  size_t bytes = 0;
  void* vhi = nullptr;  // pre-split, pre-swizzled V tiles (per k-step [hi | lo])
  void* vlo = nullptr;  // device scalars: max|V|, scale t
};
void plan_tc_project(char* base, TcProjectWs& w, int xt, int64_t n, int k);

// Serving batches: one 128-row tile of one request per table entry; all tiles
// of a launch share the X type and NPAD = k rounded up to 64.
struct TcProjUnit {
  const void* X;
  int64_t ldx;
  int64_t m;      // rows of the request
  int64_t row0;   // first row of this tile
  int64_t n;
  int32_t k;
  int32_t pad;
  const uint8_t* vt;     // V tiles of the request's V (tc_tile_v)
  const float* vscale;   // V scale (FP32 X) in the V tiles' scalar slot
  float* Y;              // m x k output of the request
};
size_t tc_tile_v_bytes(int64_t n, int k);
// Split and tile V for X type xt; scal: 2 device floats (max|V|, scale).
// exact_v: V is exact in one piece (the very sparse Omega), tiled for the exact-V products.
void tc_tile_v(Launcher& L, int xt, const float* V, int64_t n, int k, void* tiles, float* scal, int* status,
               bool exact_v = false);
// Y = X V with V already split and tiled by tc_tile_v (vscale = its scale slot).
// exact_v: V is exact in its hi piece (the very sparse Omega), so the products
// with its lo piece are skipped.  xmax / ymax (nullable): max|X| and max|Y| are
// folded into them with atomic max; NaN / Inf in X set ST_NONFINITE.
void tc_project_pretiled(Launcher& L, const void* X, int xt, int64_t m, int64_t n, int64_t ldx, const void* tiles,
                         const float* vscale, int k, float* Y, int* status, bool exact_v = false,
                         float* xmax = nullptr, float* ymax = nullptr);
// One persistent launch over *d_count (<= max_tiles) table entries.
void tc_project_batch(Launcher& L, int xt, int k, const TcProjUnit* d_units, const int* d_count, int max_tiles,
                      int* status);
// Y = X V for BF16 or E4M3 X with X fed by TMA (xproj.cu).  vtiles: V split
// and tiled by tile_v_kernel (BF16 X: BF16 pair, or the exact hi piece with
// exact_v; E4M3 X: FP16 pair of V t with t at *vscale).  check_y: a non-finite
// Y sets ST_NONFINITE.  False (nothing launched) when X's alignment or pitch
// does not allow the tensor map.
bool tc_xproj_ok(const void* X, int xt, int64_t ldx, bool exact_v);
// V split and tiled once (into w.vhi, its scale at w.vlo[1]) for several
// tc_xproj launches over row ranges of one BF16 / E4M3 X; false for other types.
bool tc_xproj_tile_v(Launcher& L, int xt, const float* V, int64_t n, int k, TcProjectWs& w, int* status);
bool tc_xproj(Launcher& L, const void* X, int xt, int64_t m, int64_t n, int64_t ldx, const void* vtiles,
              const float* vscale, int k, bool exact_v, float* Y, int* status, float* ymax, bool check_y);
void tc_project(Launcher& L, const void* X, int xt, int64_t m, int64_t n, int64_t ldx, const float* V, int k,
                TcProjectWs& w, float* Y, int* status, bool exact_v = false, float* xmax = nullptr,
                float* ymax = nullptr);

}  // namespace lspca
