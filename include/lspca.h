/*
 * lspca.h -- C ABI of the GB300 Lazy stochastic PCA library (liblspca.so).
 *
 * Method: Wojnowicz, Nguyen, Li, Zhao, "Lazy stochastic principal component
 * analysis", arXiv 1709.07175.  Notation of the paper: X is m x n with the
 * samples as rows (Sec. I-A), Omega is n x l with l = k (no oversampling, as
 * in Experiment 1; lspca_fit_oversampled takes l > k), U = X Omega (Eq. 1,
 * c = 1), F = U^T X, V is n x k, and the reduction is Y = X V (Sec. III-B.2,
 * Eq. "dim_reduction_maps").
 *
 * Conventions for every entry point
 * ---------------------------------
 * - All matrices are row-major.  A dense X has leading dimension ldx
 *   (elements, ldx >= n); ldx * sizeof(element) must be a multiple of 16
 *   bytes and X 16-byte aligned (pad rows otherwise).  A sparse X is given in
 *   CSR form (lspca_fit_csr).  V is n x k (ld k), Y is m x k
 *   (ld k), U is m x k (ld k), F is k x n (ld n), G is k x k (ld k).
 * - The "result type" of a path is FP64 when X is LSPCA_F64 and FP32
 *   otherwise; V, U and Y are stored in the result type.
 * - Pointers marked [dev] are device pointers on the context's device; the
 *   caller owns them and keeps them alive until the stream has completed.
 *   Pointers marked [host] are host pointers.
 * - Calls are asynchronous: they enqueue on `stream` (a cudaStream_t, NULL =
 *   legacy default stream) and return.  Outputs are valid after the stream
 *   has been synchronised.  Device-side failures (non-finite input, a wait
 *   that gave up) are recorded in a status word of the context; they are
 *   returned by lspca_sync_status() or by any call given a non-NULL report.
 * - No call throws; every call returns an lspca_status.  No call falls back
 *   to the host: every step runs in the library's CUDA kernels.
 * - A context serialises its workspace: calls on one context must be issued
 *   from one host thread at a time (they may use different streams only if
 *   the caller orders them).
 * - X is never centred (Sec. I-B: uncentred principal components).
 */
#ifndef LSPCA_H
#define LSPCA_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lspca_ctx lspca_ctx;

/* Return codes. */
typedef enum {
  LSPCA_OK = 0,
  LSPCA_ERR_INVALID = 1,        /* bad argument or unsupported combination      */
  LSPCA_ERR_NOMEM = 2,          /* workspace would exceed the context's budget  */
  LSPCA_WARN_RANK_DEFICIENT = 3,/* success, but rank < k (see rank rule)        */
  LSPCA_ERR_NUMERIC = 4,        /* NaN/Inf in X, or a numeric failure           */
  LSPCA_ERR_TIMEOUT = 5,        /* a bounded device or host wait gave up        */
  LSPCA_ERR_CUDA = 6,           /* a CUDA runtime/driver call failed            */
  LSPCA_ERR_BUSY = 7            /* serving: no free slot / over budget right now */
} lspca_status;

/* Element type of X (and the arithmetic the passes run in). */
typedef enum {
  LSPCA_F64 = 0,   /* FP64 SIMT throughout                                          */
  LSPCA_F32 = 1,   /* FP32 X; U in FP32; tensor-core products of exact 16-bit pieces */
  LSPCA_BF16 = 2,  /* BF16 X; BF16 tensor cores, split-BF16 U for F                 */
  LSPCA_E4M3 = 3   /* FP8 E4M3 X (binary features); needs very sparse Omega         */
} lspca_dtype;

/* The random test matrix Omega (Sec. I-A). */
typedef enum {
  LSPCA_OMEGA_GAUSSIAN = 0,     /* Omega_ij ~ N(0, 1) i.i.d.                                   */
  LSPCA_OMEGA_VERY_SPARSE = 1   /* Omega_ij in {-1, 0, +1} w.p. {1/2p, 1 - 1/p, 1/2p} (Li et al.) */
} lspca_omega_kind;

/* Omega is generated on the device from a Philox4x32-10 stream (Salmon et al.,
 * SC'11): entry (i, j) uses counter (i, j / 4, tag, 0) and key (seed mod 2^32,
 * seed / 2^32); word j % 4 feeds column j.  Gaussian (tag 0): Box-Muller on
 * word pairs (w0,w1) -> columns 4b (cos), 4b+1 (sin), (w2,w3) -> 4b+2, 4b+3,
 * u = (w + 1/2) 2^-32, FP64 then rounded to FP32 (and to BF16 on the BF16
 * path).  Very sparse (tag 1): T = floor(2^32 / 2p), w < T -> -1,
 * T <= w < 2T -> +1, else 0.  p is ignored for the Gaussian kind.          */
typedef struct {
  int32_t kind;    /* lspca_omega_kind */
  uint32_t p;      /* very sparse parameter, p >= 1 */
  uint64_t seed;
} lspca_omega;

/* Flags of the fit calls. */
enum {
  LSPCA_WANT_GRAM = 2,     /* also return G = U^T U (k x k, FP64)            */
  LSPCA_FORCE_SIMT = 16    /* run the plain SIMT kernels instead of the
                              tensor-core ones (cross-checks; slow)          */
};

/* Per-call report, filled only when a non-NULL pointer is given; the call then
 * synchronises `stream` before returning.                                    */
typedef struct {
  double ms_total;        /* host wall time of the call incl. synchronisation */
  double ms_sketch;       /* device time of pass S (U = X Omega)               */
  double ms_chain;        /* device time of pass F (F = U^T X [, G])           */
  double ms_small;        /* device time of the k x k step                     */
  double ms_qr;           /* SPCA only: TSQR and R^-T F                        */
  double bytes_x;         /* bytes of X read per pass                          */
  int32_t rank;           /* numerical rank (rank rule)                         */
  int32_t device_status;  /* status word read from the device                  */
  int32_t sweeps;         /* levels of the graded k x k eigensolve that ran (1-3) */
  int32_t qr_path;        /* SPCA's R: 1 CholeskyQR2, 2 Householder TSQR; 0 Lazy */
} lspca_report;

/* ------------------------------------------------------------------------- */

/* Create a context on `device`.  hbm_budget_bytes caps the library-owned
 * workspace (0 = 3/4 of the free device memory at creation).  The workspace
 * is allocated lazily and grown on demand up to the budget.
 * Errors: LSPCA_ERR_INVALID (out == NULL, bad device), LSPCA_ERR_CUDA.      */
int lspca_create(lspca_ctx** out, int device, size_t hbm_budget_bytes);

/* Destroy a context; synchronises its device and frees its workspace.      */
int lspca_destroy(lspca_ctx* ctx);

/* Lazy SPCA fit, Algorithm 2 / 4 (table of Sec. III):
 *   U = X Omega; F = U^T X (Alg. 4's slice sum F += U_s^T X_s over row tiles);
 *   truncated SVD of F by the eigen route of the table footnote:
 *   F F^T = W Lambda W^T, D = Lambda^1/2, V = F^T W D^-1.
 * X      [dev]  m x n, element type xt, leading dimension ldx.
 * k             target dimension, 1 <= k <= min(m, n, 256).
 * V      [dev]  n x k output in the result type: columns are the approximate right singular
 *               vectors V^l in descending sigma order; each column's largest-
 *               magnitude entry is positive; columns beyond the rank are 0.
 * sigma  [dev]  k FP64 output: singular values of U^T X (0 beyond the rank).
 * gram   [dev]  k x k FP64 output G = U^T U when flags has LSPCA_WANT_GRAM
 *               (may be NULL otherwise).
 * rank   [dev]  int32 output (nullable): numerical rank, lambda_i >
 *               max(m, n) 2^-52 lambda_1.
 * rep    [host] nullable report; non-NULL synchronises the stream.
 * Errors: LSPCA_ERR_INVALID (NULL pointers, k out of range, ldx < n,
 * misaligned X/ldx, E4M3 with a Gaussian Omega, p == 0 for very sparse),
 * LSPCA_ERR_NOMEM, LSPCA_ERR_NUMERIC (with rep: NaN/Inf found in X),
 * LSPCA_WARN_RANK_DEFICIENT (with rep), LSPCA_ERR_CUDA.                     */
int lspca_fit(lspca_ctx* ctx, const void* X, int32_t xt, int64_t m, int64_t n, int64_t ldx,
              int32_t k, lspca_omega om, uint32_t flags, void* V, double* sigma, double* gram,
              int32_t* rank, void* stream, lspca_report* rep);

/* Lazy SPCA fit of a sparse X given in CSR form (rows = samples), the format
 * of the paper's experiments (sparse slices, Sec. IV; the cost of Algorithm 2
 * is then proportional to nnz(X), Prop. 4): U = X Omega row by row
 * (compensated FP32 sums of the gathered rows of the FP32 Omega: exact
 * products, Neumaier summation; U stored in FP32),
 * F = U^T X column by column over a stable CSC copy of X built on the device
 * (every sum in a fixed order: two fits of the same input are bit-identical),
 * then the k x k step of lspca_fit.
 * row_ptr [dev]  m + 1 int64 offsets, row_ptr[0] = 0, nondecreasing,
 *                row_ptr[m] = nnz.
 * col_idx [dev]  nnz int32 column indices of the nonzeros (any order within
 *                a row; duplicates are summed).
 * val     [dev]  nnz FP32 values.
 * n              columns, 1 <= n <= 2^31 - 1.
 * k, om, V (FP32, n x k), sigma, rank, rep: as lspca_fit; flags must be 0.
 * The workspace holds Omega (n x k FP32), U (m x k FP32), F, the CSC copy (8
 * bytes per nonzero plus per-column counters of ceil(m / S) row blocks,
 * S >= 256 rows chosen to keep them near 256 MB) and the k x k step's.
 * Errors: as lspca_fit; with rep (or at lspca_sync_status) LSPCA_ERR_INVALID
 * for a column index outside [0, n) and LSPCA_ERR_NUMERIC for NaN / Inf
 * values.                                                                  */
int lspca_fit_csr(lspca_ctx* ctx, const int64_t* row_ptr, const int32_t* col_idx, const float* val, int64_t m,
                  int64_t n, int64_t nnz, int32_t k, lspca_omega om, uint32_t flags, float* V, double* sigma,
                  int32_t* rank, void* stream, lspca_report* rep);

/* The reduction map Y = X V (Sec. III-B.2) of a sparse X in CSR form (as
 * lspca_fit_csr): Y[i, :] = sum over row i's nonzeros (j, x) of x V[j, :],
 * compensated FP32 sums, Y m x k FP32 row-major.  V [dev] n x k FP32 row-major.
 * Errors: LSPCA_ERR_INVALID for bad arguments (column indices are checked on
 * the device and reported by lspca_sync_status), LSPCA_ERR_CUDA.           */
int lspca_project_csr(lspca_ctx* ctx, const int64_t* row_ptr, const int32_t* col_idx, const float* val, int64_t m,
                      int64_t n, int64_t nnz, const float* V, int32_t k, float* Y, void* stream);

/* Lazy SPCA fit with oversampling, l >= k (Sec. I-B: l = k + p with a small
 * oversampling parameter p; the Corollary of Sec. II bounds the error of the
 * l-dimensional approximation): the fit of lspca_fit with an l-column Omega
 * (its first k columns are the k-column Omega of the same seed), then the
 * truncation of the SVD of F = U^T X to its top k.  V receives the first k
 * columns (descending sigma, sign rule as lspca_fit), sigma the first k
 * values, rank min(rank of the l-column fit, k).  The span of the top-k
 * truncation depends on l and, unlike the full l-dimensional span (Prop. 2),
 * differs from SPCA's in general.
 * l             k <= l <= min(m, n, 256); l = k is lspca_fit.
 * Other arguments: as lspca_fit, with V n x k; flags must not hold
 * LSPCA_WANT_GRAM.  The n x l intermediate V and the l values of sigma live in
 * a context-owned buffer, grown on demand (a device synchronisation) and freed
 * by lspca_destroy.
 * Errors: as lspca_fit; LSPCA_ERR_INVALID also for l < k or LSPCA_WANT_GRAM;
 * with rep, LSPCA_WARN_RANK_DEFICIENT only when the rank is below k.        */
int lspca_fit_oversampled(lspca_ctx* ctx, const void* X, int32_t xt, int64_t m, int64_t n, int64_t ldx,
                          int32_t k, int32_t l, lspca_omega om, uint32_t flags, void* V, double* sigma,
                          int32_t* rank, void* stream, lspca_report* rep);

/* SPCA fit, the comparison path: Algorithm 1 in its streaming form,
 * Algorithm 3 (table of Sec. III; Eq. "approx_svd"): U = X Omega; R, the
 * triangular factor of the QR of U (Q itself is never kept, as in
 * Algorithm 3); F = R^-T U^T X (= Q^T X); truncated SVD of F by the same eigen
 * route.  R comes from CholeskyQR2 for FP32 U on the tensor-core paths:
 * R1 = chol(U^T U) from pass F's Gram, Q1 = U R1^-1 on the tensor cores,
 * R2 = chol(Q1^T Q1), R = R2 R1.  When a Cholesky meets a pivot below 1e-6
 * of its diagonal entry (U too close to rank deficient for the Gram's
 * precision) the tall-skinny Householder QR runs instead (row blocks, then a
 * reduction tree of the stacked R factors: Algorithm 3's qr([R; U_s]) in
 * parallel form); FP64 U and the SIMT paths always take it.  The report's
 * qr_path says which ran.
 * Arguments and errors as lspca_fit; sigma receives Sigma^s of Q^T X and
 * V receives V^s.  `gram` (with LSPCA_WANT_GRAM) receives U^T U.           */
int spca_fit(lspca_ctx* ctx, const void* X, int32_t xt, int64_t m, int64_t n, int64_t ldx,
             int32_t k, lspca_omega om, uint32_t flags, void* V, double* sigma, double* gram,
             int32_t* rank, void* stream, lspca_report* rep);

/* Lazy SPCA fit of a host-resident X, Algorithm 4 proper (table of Sec. III:
 * F += U_s^T X_s over row slices X_s; the paper's setting in which X does not
 * fit in memory).  The slices are copied into two device staging buffers on
 * a stream of the context while the previous slice's sketch U_s = X_s Omega
 * and F += U_s^T X_s run on `stream`; then the k x k step runs once, as in
 * lspca_fit.
 * Xh     [host] m x n, element type xt (LSPCA_F32, LSPCA_BF16 or LSPCA_E4M3),
 *               leading dimension ldx; page-locked memory (cudaHostAlloc,
 *               cudaHostRegister) lets the copies overlap the computation.
 *               Xh must stay valid and unchanged until the stream completes.
 * slice_rows    rows per slice (0 = about 256 MB of X per slice); rounded up
 *               to a multiple of 128 and capped at m.
 * k             1 <= k <= min(m, n, 256), a multiple of 4.
 * V, sigma, rank, rep: as lspca_fit (V in FP32).  flags: 0 (no Gram).
 * The workspace holds two slices, one slice of U and the k x n FP64 F, so
 * its size does not depend on m.  Slicing changes only the order in which
 * F's terms are summed (Algorithm 2 = Algorithm 4 up to rounding).
 * Errors: as lspca_fit; LSPCA_ERR_INVALID also for F64 X, k not a multiple
 * of 4, LSPCA_WANT_GRAM / LSPCA_FORCE_SIMT in flags, or no sm_103 device.    */
int lspca_fit_host(lspca_ctx* ctx, const void* Xh, int32_t xt, int64_t m, int64_t n, int64_t ldx, int32_t k,
                   lspca_omega om, uint32_t flags, int64_t slice_rows, void* V, double* sigma, int32_t* rank,
                   void* stream, lspca_report* rep);

/* Fit and reduction map of a host-resident X in one call, the whole step of
 * Experiment 1 from host memory (Algorithm 4 for the fit, Sec. III-B.2 for
 * Y = X V): X is copied in row slices on a second stream into Xd while each
 * slice already copied is sketched and folded into F, as in lspca_fit_host;
 * after the k x k step, Y is computed slice by slice (slices of about 128 MB
 * of Y) into two device staging buffers, and each slice is copied back into
 * Yh while the next one is projected.
 * Xh [host] m x n (xt F32, BF16 or E4M3; pinned memory for overlapped
 * copies), ldx as in lspca_fit; Xd [dev] m x ldx elements of xt, 16-byte
 * aligned, owned by the caller, receives X (and keeps it); V [dev] n x k FP32,
 * sigma [dev] k FP64, rank [dev] nullable, outputs as in lspca_fit; Yh [host]
 * m x k FP32 output (pinned memory for overlapped copies).  k a multiple of 4,
 * slice_rows and flags as lspca_fit_host.  Everything is asynchronous on
 * `stream`: Yh is complete when the stream has completed.  With rep, ms_qr
 * holds the time of the reduction map and its copies.
 * Errors: as lspca_fit_host; LSPCA_ERR_INVALID also for NULL Xd or Yh or a
 * misaligned Xd.                                                           */
int lspca_fit_project_host(lspca_ctx* ctx, const void* Xh, int32_t xt, int64_t m, int64_t n, int64_t ldx, int32_t k,
                           lspca_omega om, uint32_t flags, int64_t slice_rows, void* Xd, void* V, double* sigma,
                           int32_t* rank, float* Yh, void* stream, lspca_report* rep);

/* Reduction map pi(x) = V^T x for every row: Y = X V (Sec. III-B.2).
 * X [dev] m x n (xt, ldx); V [dev] n x k and Y [dev] m x k (output), both
 * in the result type.  F32 X, k <= 128: X and V each split into three exact
 * BF16 pieces (x = x0 + x1 + x2), the six products x_a v_b with a + b <= 2;
 * F32 X, k > 128: FP16 pairs (hi + lo, power-of-two scales), three products;
 * BF16/E4M3 X: V split into a BF16 pair, two products; F64 X: FP64 SIMT.
 * 1 <= k <= 256.
 * Errors: LSPCA_ERR_INVALID, LSPCA_ERR_NOMEM, LSPCA_ERR_CUDA.               */
int lspca_project(lspca_ctx* ctx, const void* X, int32_t xt, int64_t m, int64_t n, int64_t ldx,
                  const void* V, int32_t k, void* Y, void* stream);

/* ---- step-level entry points (the passes of lspca_fit, for tests) ----- */

/* Write Omega (n x k row-major) as generated on the device.  t selects the
 * output element type: LSPCA_F64 (the FP32-rounded values, or exact +-1/0),
 * LSPCA_F32, or LSPCA_BF16 (BF16-rounded, as the BF16 path uses it).
 * out [dev].  Errors: LSPCA_ERR_INVALID, LSPCA_ERR_CUDA.                    */
int lspca_omega_materialize(lspca_ctx* ctx, lspca_omega om, int64_t n, int32_t k, int32_t t,
                            void* out, void* stream);

/* Pass S: U = X Omega (Eq. 1, c = 1; Algorithm 2 step 1).  U [dev] m x k,
 * FP64 when xt == LSPCA_F64, else FP32.  Errors as lspca_fit.               */
int lspca_sketch(lspca_ctx* ctx, const void* X, int32_t xt, int64_t m, int64_t n, int64_t ldx,
                 int32_t k, lspca_omega om, uint32_t flags, void* U, void* stream);

/* Pass F: F = U^T X (Algorithm 2 step 2; Algorithm 4's slice sum) and, when
 * G != NULL, G = U^T U.  U [dev] m x k (FP64 if xt == LSPCA_F64, else FP32);
 * F [dev] k x n FP64; G [dev] k x k FP64 or NULL.                           */
int lspca_chain(lspca_ctx* ctx, const void* X, int32_t xt, int64_t m, int64_t n, int64_t ldx,
                const void* U, int32_t k, uint32_t flags, double* F, double* G, void* stream);

/* The k x k step (table footnote): H = F F^T, H = W Lambda W^T (descending),
 * sigma = Lambda^1/2, V = F^T W D^-1, sign and rank rules as lspca_fit.
 * F [dev] k x n FP64; V [dev] n x k output, FP64 when vt == LSPCA_F64, FP32
 * when vt == LSPCA_F32; sigma [dev] k FP64; rank [dev] nullable; m is the
 * row count of X (used by the rank rule only).                             */
int lspca_decompose(lspca_ctx* ctx, const double* F, int32_t k, int64_t n, int64_t m, int32_t vt, void* V,
                    double* sigma, int32_t* rank, void* stream);

/* Pass F without any allocation (the paper has no counterpart: this serves
 * callers that may not allocate device memory, e.g. code running inside a
 * framework that owns all GPU memory through its own pool, or loops that
 * cannot afford the device synchronisation cudaMalloc/cudaFree imply).
 * Computes F = U^T X with the same split-product arithmetic as lspca_chain's
 * tensor-core path (FP32 X: FP16 pairs; BF16 X: U as a BF16 pair) but in its
 * own kernel and chunking, so the two agree within pass F's tolerance, not
 * bit for bit; no context is needed.
 * X [dev] m x n, xt LSPCA_F32 or LSPCA_BF16; U [dev] m x k FP32 (ld k);
 * 4 <= k <= 256, k a multiple of 4; F [dev] k x n FP64 output;
 * status [dev] int32 output (nullable): zeroed, then the device status bits
 * (1 = NaN or Inf in X, 2 = a bounded wait inside the kernel gave up);
 * stream as elsewhere.
 * Scratch: a 16 MiB device array inside the library, held by every GPU that
 * loads the library until the process exits; k * n * 4 bytes of it must hold
 * one chunk's partial sums (k * n <= 4,194,240), else LSPCA_ERR_NOMEM.  The
 * first call on a device looks up the array's device address, so make it
 * before any stream capture.  Every call shares the array: calls whose
 * executions overlap on the GPU race on it and must be ordered by the caller.
 * Allocates nothing (no cudaMalloc, cudaFree or allocating library call).
 * Errors: LSPCA_ERR_INVALID (NULL or misaligned pointers, k or xt out of
 * range, no sm_103 device), LSPCA_ERR_NOMEM (k * n too large), LSPCA_ERR_CUDA. */
int lspca_chain_noalloc(const void* X, int32_t xt, int64_t m, int64_t n, int64_t ldx, const float* U, int32_t k,
                        double* F, int32_t* status, void* stream);

/* ---- serving: continuous batching (a request loop on one GPU) ----------
 * Not in the paper: a runtime that keeps fitted V matrices resident and
 * serves reduction-map requests (Y = X V, Sec. III-B.2) and Lazy SPCA fits
 * (Algorithm 4, one slice of 65,536 rows per step) submitted while others
 * run.  All buffers passed in are device memory owned by the caller and must
 * stay valid until the request is done.
 *
 * lspca_srv_create: server on `device` with its own stream and an HBM arena
 *   of hbm_budget_bytes (0 = 4 GiB) for fit workspaces and V tiles;
 *   max_inflight bounds the requests admitted at once.
 * lspca_srv_register_v: keep V (n x k FP32, row-major, 4 <= k <= 256, k a
 *   multiple of 4) for projection requests; returns its id.
 * lspca_srv_submit_project: queue Y[rows x k] = X[rows x n] V (X FP32, BF16
 *   or E4M3 with leading dimension ldx).
 * lspca_srv_submit_fit: queue a Lazy SPCA fit of X (m x n, FP32/BF16/E4M3)
 *   into V (n x k FP32) and sigma (k FP64); LSPCA_ERR_NOMEM if its workspace
 *   can never fit the arena.
 * lspca_srv_step: admit queued requests in FIFO order while a slot is free and
 *   (for fits) the workspace fits the arena, then launch one batch: all
 *   running projections' 128-row tiles in one table-driven launch per (X type,
 *   padded k) -- replayed as a captured CUDA graph -- and one slice of every
 *   running fit.  work_units (nullable) receives tiles + fit slices launched.
 * lspca_srv_poll: done = 1 once the request's results are complete on the GPU.
 * lspca_srv_wait: drive steps / wait until done or timeout_ms elapsed
 *   (LSPCA_ERR_TIMEOUT).
 * lspca_srv_release: forget a finished request (LSPCA_ERR_BUSY if not done).
 * Each request's arithmetic depends only on the request (fixed tiles and
 * slices), so its results are bit-identical alone and in any mix.            */
typedef struct lspca_srv lspca_srv;
int lspca_srv_create(lspca_srv** out, int device, size_t hbm_budget_bytes, int32_t max_inflight);
int lspca_srv_destroy(lspca_srv* srv);
int lspca_srv_register_v(lspca_srv* srv, const float* V, int64_t n, int32_t k, int32_t* v_id);
int lspca_srv_submit_project(lspca_srv* srv, int32_t v_id, const void* X, int32_t xt, int64_t rows, int64_t ldx,
                             float* Y, int64_t* req);
int lspca_srv_submit_fit(lspca_srv* srv, const void* X, int32_t xt, int64_t m, int64_t n, int64_t ldx, int32_t k,
                         lspca_omega om, float* V, double* sigma, int64_t* req);
int lspca_srv_step(lspca_srv* srv, int32_t* work_units);
int lspca_srv_poll(lspca_srv* srv, int64_t req, int32_t* done);
int lspca_srv_wait(lspca_srv* srv, int64_t req, int32_t timeout_ms);
int lspca_srv_release(lspca_srv* srv, int64_t req);
int64_t lspca_srv_launch_count(lspca_srv* srv);

/* Fixed-order sum of gathered partials, the exchange of a row-sharded fit
 * (Algorithm 4's F = sum_s U_s^T X_s with the slices spread over ranks, and
 * likewise G = sum_s U_s^T U_s): out[e] = (((p_0[e] + p_1[e]) + p_2[e]) + ...)
 * in FP64, p_q[e] = parts[q * count + e].  Every rank that calls it on the
 * same gathered parts holds the same bits, whatever order the collective used.
 * parts [dev] nparts x count FP64; out [dev] count FP64 (may not overlap parts).
 * Errors: LSPCA_ERR_INVALID (NULL pointers, nparts < 1, count < 0),
 * LSPCA_ERR_CUDA.                                                          */
int lspca_sum_partials(lspca_ctx* ctx, const double* parts, int32_t nparts, int64_t count, double* out,
                       void* stream);

/* The failure path of the device waits, run on purpose: one CTA waits, with
 * the time-limited mbarrier wait every tensor-core pipeline uses, on a barrier
 * that no thread arrives at.  After limit_ns nanoseconds (%globaltimer) the
 * wait gives up, sets the timeout bit of the context's status word and raises
 * the CTA's abort flag; the CTA's other warps leave their polling loops and
 * the kernel ends normally, as a pipeline's roles do.  The next
 * lspca_sync_status returns LSPCA_ERR_TIMEOUT and the context stays usable.
 * Not in the paper: it tests the library's error handling.
 * waited_ns [dev, nullable] int64 output: how long the wait lasted.
 * Errors: LSPCA_ERR_INVALID (NULL ctx, limit_ns outside [1e3, 2e9]),
 * LSPCA_ERR_CUDA.                                                          */
int lspca_wait_probe(lspca_ctx* ctx, int64_t limit_ns, int64_t* waited_ns, void* stream);

/* Synchronise `stream`, return and clear the device status word:
 * LSPCA_OK, LSPCA_ERR_NUMERIC or LSPCA_ERR_TIMEOUT.                         */
int lspca_sync_status(lspca_ctx* ctx, void* stream);

/* Human-readable text of a status code (static storage).                   */
const char* lspca_strerror(int status);

/* Number of kernels this library has launched on this context (a counter
 * kept by the host side; used to report launch counts).                    */
int64_t lspca_launch_count(lspca_ctx* ctx);

/* Pass timing without synchronisation: with profiling enabled every fit
 * records CUDA events between its kernels on its stream (up to 4096 calls
 * are kept); lspca_profile_read synchronises the device and returns the
 * summed device milliseconds ms7[0..6] = {Omega generation (+ X scan),
 * pass-S kernel, pass-F main kernel, pass-F reduction, SPCA QR + R^-T F,
 * k x k step, whole call} and the number of calls.  enable = 0 stops and
 * resets.                                                                   */
int lspca_profile(lspca_ctx* ctx, int enable);
int lspca_profile_read(lspca_ctx* ctx, double* ms7, int64_t* calls);

#ifdef __cplusplus
}
#endif
#endif /* LSPCA_H */
