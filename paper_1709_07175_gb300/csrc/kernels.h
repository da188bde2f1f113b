// Host-side launchers of liblspca's kernels (internal interface between the
// C-ABI layer and the kernel translation units).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/lspca.h"

namespace lspca {

struct Launcher {
  cudaStream_t stream;
  int64_t* counter;
  int num_sms;
  void count(int n) { *counter += n; }
};

// Launch with programmatic stream serialization (the kernel must start with
// pdl_wait(); see common.cuh): its launch overlaps the predecessor's run.
template <typename... KArgs, typename... Args>
inline void launch_pdl(Launcher& L, void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem, Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = L.stream;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  cudaLaunchKernelEx(&cfg, kern, static_cast<KArgs>(args)...);
}

// ---- K0: Omega ------------------------------------------------------------
void launch_omega_dense(Launcher& L, const lspca_omega& om, int64_t n, int k, int out_dt, void* out, int64_t ld,
                        bool transposed, bool bf16_round);
void launch_omega_csc(Launcher& L, const lspca_omega& om, int64_t n, int k, int32_t* counts, int32_t* col_ptr,
                      int32_t* entries);

// ---- generic SIMT GEMM ------------------------------------------------------
// C[s][M x N] = sum over K-range s of op(A) op(B), one partial per split s
// (stride c_split_stride).  op(A)(r, kk) = a_trans ? A[kk*lda + r] : A[r*lda + kk],
// op(B)(kk, c) = b_trans ? B[c*ldb + kk] : B[kk*ldb + c].
// Element types: ta/tb in {F64, F32, BF16, E4M3} (lspca_dtype); acc_f64 selects
// FP64 accumulation; c_f64 selects an FP64 (else FP32) output.
void launch_gemm_simt(Launcher& L, int64_t M, int64_t N, int64_t K, const void* A, int ta, int64_t lda, bool a_trans,
                      const void* B, int tb, int64_t ldb, bool b_trans, void* C, bool c_f64, int64_t ldc,
                      int64_t c_split_stride, int splits, bool acc_f64, bool small_tiles);

// out[e] = sum_{s < splits} part[s * stride + e] in FP64, fixed order; count elements.
void launch_reduce_splits(Launcher& L, const double* part, int splits, int64_t stride, int64_t count, double* out);

// ---- K1: pass S -----------------------------------------------------------
// U = X Omega with very sparse Omega (CSC lists); U is FP64 for F64 X, else FP32.
// absmax[0] |= max|X|, absmax[1] |= max|U| (FP32 bit-pattern max); status |= ST_NONFINITE.
// `off` is a k x (chunks + 1) int32 scratch (sketch_off_bytes) used when the
// per-(column, chunk) offset table does not fit in shared memory.
size_t sketch_off_bytes(int64_t n, int k);
void launch_sketch_sparse(Launcher& L, const void* X, int xt, int64_t m, int64_t n, int64_t ldx, int k,
                          const int32_t* col_ptr, const int32_t* entries, int32_t* off, void* U, int64_t ldu,
                          float* absmax, int* status);
// U = X Omega for FP8 E4M3 X and the very sparse Omega, as a gather over the
// nonzeros of X (bsketch.cu); ws holds Omega's rows (bsketch_ws_bytes).  U is
// m x k FP32; *umax |= max|U|; NaN in X sets ST_NONFINITE.
size_t bsketch_ws_bytes(int64_t n, int k);
void launch_bsketch(Launcher& L, const void* X, int64_t m, int64_t n, int64_t ldx, int k, const lspca_omega& om,
                    void* ws, float* U, float* umax, int* status);
// FP8 tensor-core passes for E4M3 X with the very sparse Omega (f8.cu).  One
// workspace (f8_ws_bytes) serves both: the sketch writes U (FP32, nullable)
// and its E4M3 copy plus a flag raised when some U is not exactly an E4M3
// value; pass F (launch_f8_chain: F = U^T X, k x n FP64) then reads the E4M3
// copy, or does nothing when the flag is raised (f8_inexact_flag: the gate of
// the BF16 pass F that runs instead).  launch_f8_u8 makes the copy of a
// caller-supplied U.  The launchers return false when a tensor map cannot be
// built.
size_t f8_ws_bytes(int64_t m, int64_t n, int k, int num_sms);
int* f8_inexact_flag(void* ws, int64_t m, int64_t n, int k, int num_sms);
// U (FP32) is nullable: the E4M3 copy alone feeds the FP8 pass F.  again:
// the run after one with U == nullptr, which writes U only if that run found U
// not exact in E4M3 (the BF16 pass F then needs it); it does nothing otherwise.
bool launch_f8_sketch(Launcher& L, const void* X, int64_t m, int64_t n, int64_t ldx, int k, const lspca_omega& om,
                      void* ws, float* U, float* umax, int* status, bool again = false);
void launch_f8_u8(Launcher& L, const float* U, int64_t m, int k, void* ws, int64_t n);
bool launch_f8_chain(Launcher& L, const void* X, int64_t m, int64_t n, int64_t ldx, int k, void* ws, double* F,
                     int* status);
// Scan X for NaN/Inf and its largest magnitude (dense-Omega paths).
void launch_scan_x(Launcher& L, const void* X, int xt, int64_t m, int64_t n, int64_t ldx, float* absmax, int* status);

// ---- K3: the k x k step ---------------------------------------------------
// ---- sparse X (CSR, rows = samples) ------------------------------------------
// Y[i, :] = sum over row i's nonzeros (j, x) of x D[j, :] (D n x k FP32,
// compensated FP32 sums, Y m x k FP32): the sketch with D = Omega, the
// reduction map with D = V.
void launch_csr_rows(Launcher& L, const int64_t* row_ptr, const int32_t* col, const float* val, int64_t m, int64_t n,
                     int64_t nnz, const float* D, int k, float* Y, int* status);
// Stable CSR -> CSC (entries of a column in row order) in the workspace `ws`
// of csc_ws_bytes bytes, which also holds pass F's segment partials.
struct CscView {
  int64_t* col_ptr;   // n + 1
  int32_t* crow;      // nnz row indices
  float* cval;        // nnz values
  int64_t* segc;      // n: segments per column
  int64_t* seg_ptr;   // n + 1
  double* part;       // max_segments x k partials of F
  int64_t max_segments;
};
int64_t csr_rows_per_block(int64_t m, int64_t n);
size_t csc_ws_bytes(int64_t m, int64_t n, int64_t nnz, int k);
void launch_csr_to_csc(Launcher& L, const int64_t* row_ptr, const int32_t* col, const float* val, int64_t m,
                       int64_t n, int64_t nnz, int k, void* ws, CscView* out);
// F[:, j] = sum over column j's entries (row order) of x U[i, :]; F k x n FP64.
void launch_csc_passf(Launcher& L, const CscView& c, int64_t n, int64_t nnz, const float* U, int k, double* F);

struct SmallWs {
  double* Hpart;   // splits x k x k
  void* oz;        // workspace of the tensor-core H = F F^T (ozaki.cu)
  double* H;       // k x k
  float* h32;      // k x k: the seed's tridiagonalisation reflectors
  float* w32;      // k x k: the seed's eigenvectors of T (column-major)
  float* q32;      // k x k: inverse-iteration pivots, then Householder vectors
  float* p32;      // k x k: working copy of the seed's Householder QR
  double* Xa;      // k x k
  double* Xb;      // k x k
  double* Rm;      // k x k
  double* T;       // k x k
  double* S;       // k x k
  double* E;       // k x k
  double* lam;     // k
  double* scal;    // 8 scalars, sigma copy (k), sqrt(S_rr) (k), order (k int32)
  double* Vd;      // n x k
  void* vaux;      // FP32 V: per-tile column maxima, column signs, tile counters
  int32_t* sweeps; // 1: levels of the graded eigen seed that ran
  int32_t* lvl;    // kSeedLevels + 1: block size of each seed level
  int32_t* cid;    // k: seed cluster of each eigenvector column (level * 1024 + cluster)
  float* tri;      // seed scratch: d, e, e^2, beta, eigenvalues of T (k each), 8 scalars
  int h_splits;
};
// Levels of the graded eigensolve of the k x k step (eigseed.cu).
constexpr int kSeedLevels = 3;
size_t small_ws_bytes(int k, int64_t n, int* h_splits);
// One level of the FP32 eigen seed (eigseed.cu).  Level 0 seeds M = H
// (k x k FP64) and writes its eigenvectors to Xout; level l > 0 seeds the
// leading lvl[l] x lvl[l] block of M (ld k) and writes blockdiag(W, I) to
// Xout.  lvl[l + 1] receives the size of the level's unresolved tail.
// cid[i] (i < the level's block size) receives the seed cluster of column i:
// columns with equal ids were not resolved from one another by the seed.
void launch_seed_level(Launcher& L, const double* M, int k, int level, int32_t* lvl, float* gV, float* Zc, float* U,
                       float* Wk, float* tri, double* Xout, double* lam, double* scal, int32_t* stats,
                       int32_t* cid);
void carve_small_ws(SmallWs& w, void* base, int k, int64_t n);
// H = F F^T (F k x n FP64, row-major; k <= 256) on the BF16 tensor cores from
// exact digit planes of F, summed in integers (ozaki.cu): the FP64 result up
// to one final rounding and digits below 2^-57 of each row's largest entry.
size_t oz_gram_ws_bytes(int k, int64_t n);
void launch_oz_gram(Launcher& L, const double* F, int k, int64_t n, void* ws, double* H, int* status);
void launch_decompose(Launcher& L, SmallWs& w, const double* F, int k, int64_t n, int64_t m, bool v_f64, void* V,
                      double* sigma, int32_t* rank, int* status);

// ---- K4: TSQR (SPCA) ------------------------------------------------------
size_t tsqr_ws_bytes(int64_t m, int k);
// R (k x k FP64, upper triangular) of U (m x k, FP64 if u_f64 else FP32) by
// Householder reflections.  run_if (nullable): every kernel does nothing
// unless *run_if != 0 (the fallback of CholeskyQR2).
void launch_tsqr(Launcher& L, const void* U, bool u_f64, int64_t m, int k, void* ws, double* R,
                 const int* run_if = nullptr);
// CholeskyQR2 pieces (cholqr.cu); each does nothing once *fail is set.
// launch_chol: R (k x k FP32, upper) with G = R^T R, or *fail = 1 when a
// pivot falls below its tolerance.  launch_tri_inv: Rinv = R^-1 (zeros once
// *fail is set).  launch_rmul: R = R2 R1 in FP64.
size_t cholqr_smem_bytes(int k);
void launch_chol(Launcher& L, const double* G, int k, float* R, int* fail);
void launch_tri_inv(Launcher& L, const float* R, int k, float* Rinv, const int* fail);
void launch_rmul(Launcher& L, const float* R2, const float* R1, int k, double* R, const int* fail);
// F <- R^-T F in place (F k x n FP64); pivots below 1e-10 (FP64 U) or 1e-4
// (FP32 U) of the largest give zero rows.
void launch_trsm_rt(Launcher& L, const double* R, int k, double* F, int64_t n, bool u_f64);

// The bounded-wait failure path on a barrier that never completes (waitprobe.cu).
void launch_wait_probe(Launcher& L, uint64_t limit_ns, int* status, int64_t* waited_ns);

}  // namespace lspca
