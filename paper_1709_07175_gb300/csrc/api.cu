// C ABI of liblspca: context, workspace, argument checks and the orchestration of
// the passes (declared in include/lspca.h).
#include <chrono>
#include <functional>
#include <cstdint>
#include <cstring>
#include <vector>

#include "common.cuh"
#include "kernels.h"
#include "tc.h"

using namespace lspca;

struct lspca_ctx {
  int device = 0;
  size_t budget = 0;
  void* ws = nullptr;
  size_t ws_size = 0;
  int* d_status = nullptr;    // device status word
  float* d_absmax = nullptr;  // [0] max|X|, [1] max|U|
  int32_t* d_rank = nullptr;  // rank when the caller passes none
  int64_t launches = 0;
  int num_sms = 0;
  cudaEvent_t ev[6] = {};
  // host-resident fits: copy stream, per staging buffer "copied" / "consumed" events
  cudaStream_t cstream = nullptr;
  cudaEvent_t copied[2] = {};
  cudaEvent_t consumed[2] = {};
  // oversampled fits: the n x l V, the l sigma and the rank of the l-column fit
  void* aux = nullptr;
  size_t aux_size = 0;
  // profiling ring: 5 events per call
  bool profiling = false;
  std::vector<cudaEvent_t> pev;
  int64_t pcalls = 0;
};

namespace {

// Bump allocator over the context workspace (256-byte aligned pieces).
struct Plan {
  char* base = nullptr;
  size_t off = 0;
  void* take(size_t bytes) {
    off = (off + 255) & ~(size_t)255;
    void* p = base ? base + off : nullptr;
    off += bytes;
    return p;
  }
};

int cuda_status(cudaError_t e) { return e == cudaSuccess ? LSPCA_OK : LSPCA_ERR_CUDA; }

int ensure_ws(lspca_ctx* ctx, size_t bytes, cudaStream_t stream) {
  if (bytes > ctx->budget) return LSPCA_ERR_NOMEM;
  if (bytes <= ctx->ws_size) return LSPCA_OK;
  cudaError_t e = cudaStreamSynchronize(stream);
  if (e != cudaSuccess) return LSPCA_ERR_CUDA;
  if (ctx->ws) cudaFree(ctx->ws);
  ctx->ws = nullptr;
  ctx->ws_size = 0;
  size_t want = bytes + bytes / 4;
  if (want > ctx->budget) want = ctx->budget;
  e = cudaMalloc(&ctx->ws, want);
  if (e != cudaSuccess) {
    cudaGetLastError();
    e = cudaMalloc(&ctx->ws, bytes);
    if (e != cudaSuccess) {
      cudaGetLastError();
      ctx->ws = nullptr;
      return LSPCA_ERR_NOMEM;
    }
    want = bytes;
  }
  ctx->ws_size = want;
  return LSPCA_OK;
}

bool aligned16(const void* p) { return ((uintptr_t)p & 15u) == 0; }

int check_x(const void* X, int xt, int64_t m, int64_t n, int64_t ldx) {
  if (!X) return LSPCA_ERR_INVALID;
  if (xt < LSPCA_F64 || xt > LSPCA_E4M3) return LSPCA_ERR_INVALID;
  if (m < 1 || n < 1 || ldx < n) return LSPCA_ERR_INVALID;
  if (!aligned16(X) || (ldx * (int64_t)dtype_size(xt)) % 16 != 0) return LSPCA_ERR_INVALID;
  return LSPCA_OK;
}

int check_omega(const lspca_omega& om, int xt) {
  if (om.kind != LSPCA_OMEGA_GAUSSIAN && om.kind != LSPCA_OMEGA_VERY_SPARSE) return LSPCA_ERR_INVALID;
  if (om.kind == LSPCA_OMEGA_VERY_SPARSE && om.p == 0) return LSPCA_ERR_INVALID;
  if (xt == LSPCA_E4M3 && om.kind != LSPCA_OMEGA_VERY_SPARSE) return LSPCA_ERR_INVALID;
  return LSPCA_OK;
}

size_t acc_size(int xt) { return xt == LSPCA_F64 ? 8 : 4; }
int acc_dt(int xt) { return xt == LSPCA_F64 ? LSPCA_F64 : LSPCA_F32; }

double ev_ms(cudaEvent_t a, cudaEvent_t b) {
  float ms = 0.f;
  if (cudaEventElapsedTime(&ms, a, b) != cudaSuccess) {
    cudaGetLastError();
    return 0.0;
  }
  return (double)ms;
}

// ---- pass S -----------------------------------------------------------------
struct SketchBufs {
  int32_t* counts = nullptr;
  int32_t* col_ptr = nullptr;
  int32_t* entries = nullptr;
  int32_t* off = nullptr;
  void* omega = nullptr;  // dense Omega (n x k, result type) for the SIMT / tensor-core paths
  TcProjectWs pw;         // tensor-core path: pre-split tiles of Omega
  void* bsws = nullptr;   // E4M3 X, plain SIMT path: Omega's rows for the gather
  void* f8ws = nullptr;   // E4M3 X on the FP8 tensor cores (shared with pass F)
};

// FP8 E4M3 X (binary features; the very sparse Omega is required): the FP8
// tensor-core sketch and pass F (f8.cu); under LSPCA_FORCE_SIMT the sketch is
// the gather over the nonzeros of X (bsketch.cu).
bool use_f8(int xt, uint32_t flags) {
  return xt == LSPCA_E4M3 && !(flags & LSPCA_FORCE_SIMT) && tc_available();
}
bool use_bsketch(int xt, uint32_t flags) { return xt == LSPCA_E4M3 && !use_f8(xt, flags); }

void plan_sketch(Plan& P, SketchBufs& b, int xt, int64_t n, int k, const lspca_omega& om, bool tc, uint32_t flags,
                 int64_t m, int num_sms) {
  if (use_f8(xt, flags)) {
    b.f8ws = P.take(f8_ws_bytes(m, n, k, num_sms));
  } else if (use_bsketch(xt, flags)) {
    b.bsws = P.take(bsketch_ws_bytes(n, k));
  } else if (tc) {
    b.omega = P.take((size_t)n * k * 4);
    char* base = P.base ? P.base + ((P.off + 255) & ~(size_t)255) : nullptr;
    plan_tc_project(base, b.pw, xt, n, k);
    P.take(b.pw.bytes);
  } else if (om.kind == LSPCA_OMEGA_VERY_SPARSE) {
    b.counts = (int32_t*)P.take((size_t)k * 4);
    b.col_ptr = (int32_t*)P.take((size_t)(k + 1) * 4);
    b.entries = (int32_t*)P.take((size_t)n * k * 4);
    b.off = (int32_t*)P.take(sketch_off_bytes(n, k));
  } else {
    b.omega = P.take((size_t)n * k * acc_size(xt));
  }
}

using Mark = std::function<void(int)>;

// need_u: the fit uses the FP32 U itself (SPCA's QR, the Gram); otherwise the
// FP8 path writes only the E4M3 copy, and a gated second run writes U in the
// rare case that copy is not exact (the BF16 pass F then takes over).
void run_sketch(lspca_ctx* ctx, Launcher& L, const void* X, int xt, int64_t m, int64_t n, int64_t ldx, int k,
                const lspca_omega& om, bool tc, SketchBufs& b, void* U, const Mark& mark, bool need_u = true) {
  if (b.f8ws) {
    mark(1);
    launch_f8_sketch(L, X, m, n, ldx, k, om, b.f8ws, need_u ? (float*)U : nullptr, ctx->d_absmax + 1, ctx->d_status);
    if (!need_u) launch_f8_sketch(L, X, m, n, ldx, k, om, b.f8ws, (float*)U, ctx->d_absmax + 1, ctx->d_status, true);
    mark(2);
    return;
  }
  if (b.bsws) {
    mark(1);
    launch_bsketch(L, X, m, n, ldx, k, om, b.bsws, (float*)U, ctx->d_absmax + 1, ctx->d_status);
    mark(2);
    return;
  }
  if (tc) {
    // dense Omega (BF16-rounded for BF16 X, exact +-1/0 for the very sparse kind)
    // through the tensor-core reduction-map kernel: U = X Omega; the kernel also
    // takes max|X| (NaN / Inf detection) and max|U| as it streams
    launch_omega_dense(L, om, n, k, LSPCA_F32, b.omega, k, false, xt == LSPCA_BF16);
    mark(1);
    tc_project(L, X, xt, m, n, ldx, (const float*)b.omega, k, b.pw, (float*)U, ctx->d_status,
               om.kind == LSPCA_OMEGA_VERY_SPARSE, ctx->d_absmax, ctx->d_absmax + 1);
    mark(2);
    return;
  }
  if (om.kind == LSPCA_OMEGA_VERY_SPARSE) {
    launch_omega_csc(L, om, n, k, b.counts, b.col_ptr, b.entries);
    mark(1);
    launch_sketch_sparse(L, X, xt, m, n, ldx, k, b.col_ptr, b.entries, b.off, U, k, ctx->d_absmax, ctx->d_status);
    mark(2);
    return;
  }
  const bool bf = xt == LSPCA_BF16;
  launch_omega_dense(L, om, n, k, acc_dt(xt), b.omega, k, false, bf);
  launch_scan_x(L, X, xt, m, n, ldx, ctx->d_absmax, ctx->d_status);
  mark(1);
  launch_gemm_simt(L, m, k, n, X, xt, ldx, false, b.omega, acc_dt(xt), k, false, U, xt == LSPCA_F64, k, 0, 1,
                   xt == LSPCA_F64, false);
  mark(2);
}

// ---- pass F -----------------------------------------------------------------
struct ChainBufs {
  double* Fpart = nullptr;
  double* Gpart = nullptr;
  int f_splits = 1, g_splits = 1;
  TcChainWs tcw;
  void* f8ws = nullptr;  // E4M3 X: the FP8 pass F (the BF16 one runs only when U is not exact in E4M3)
};

int simt_splits(int64_t rows, int64_t cols, int64_t K, int num_sms) {
  const int64_t tiles = ((rows + 63) / 64) * ((cols + 63) / 64);
  int64_t s = (2 * num_sms + tiles - 1) / tiles;
  if (s > 64) s = 64;
  if (s > K / 64) s = K / 64;
  if (s < 1) s = 1;
  return (int)s;
}

void plan_chain(Plan& P, ChainBufs& b, int xt, int64_t m, int64_t n, int k, bool want_g, bool tc, int num_sms) {
  if (tc) {
    plan_tc_chain(P.base ? P.base + ((P.off + 255) & ~(size_t)255) : nullptr, b.tcw, xt, m, n, k, want_g, num_sms);
    P.take(b.tcw.bytes);
    return;
  }
  b.f_splits = simt_splits(k, n, m, num_sms);
  b.Fpart = (double*)P.take((size_t)b.f_splits * k * n * 8);
  if (want_g) {
    b.g_splits = simt_splits(k, k, m, num_sms);
    b.Gpart = (double*)P.take((size_t)b.g_splits * k * k * 8);
  }
}

int run_chain(lspca_ctx* ctx, Launcher& L, const void* X, int xt, int64_t m, int64_t n, int64_t ldx, const void* U,
              int k, bool tc, ChainBufs& b, double* F, double* G, const Mark& mark) {
  if (tc) {
    const int* gate = nullptr;
    if (b.f8ws) {
      if (!launch_f8_chain(L, X, m, n, ldx, k, b.f8ws, F, ctx->d_status)) return LSPCA_ERR_CUDA;
      gate = f8_inexact_flag(b.f8ws, m, n, k, ctx->num_sms);
    }
    if (!tc_chain_main(L, X, xt, m, n, ldx, (const float*)U, k, b.tcw, ctx->d_absmax, ctx->d_status, G != nullptr,
                       gate))
      return LSPCA_ERR_CUDA;
    mark(3);
    tc_chain_reduce(L, n, k, b.tcw, F, G, false, gate);
    mark(4);
    return LSPCA_OK;
  }
  const bool f64 = xt == LSPCA_F64;
  launch_gemm_simt(L, k, n, m, U, acc_dt(xt), k, true, X, xt, ldx, false, b.Fpart, true, n, (int64_t)k * n, b.f_splits,
                   f64, false);
  if (G)
    launch_gemm_simt(L, k, k, m, U, acc_dt(xt), k, true, U, acc_dt(xt), k, false, b.Gpart, true, k, (int64_t)k * k,
                     b.g_splits, f64, false);
  mark(3);
  launch_reduce_splits(L, b.Fpart, b.f_splits, (int64_t)k * n, (int64_t)k * n, F);
  if (G) launch_reduce_splits(L, b.Gpart, b.g_splits, (int64_t)k * k, (int64_t)k * k, G);
  mark(4);
  return LSPCA_OK;
}

bool use_tc_chain(int xt, uint32_t flags, int k = 4) {
  return !(flags & LSPCA_FORCE_SIMT) && xt != LSPCA_F64 && (k % 4) == 0 && tc_available();
}
// The sketch of FP32 / BF16 / E4M3 X runs on the tensor-core reduction-map
// kernel with Omega as its right operand (the very sparse Omega is exact in
// one FP16 / BF16 piece, so half the products drop out); the gather kernel of
// the very sparse Omega stays for FP64 X and under LSPCA_FORCE_SIMT.
bool use_tc_sketch(int xt, const lspca_omega& om, uint32_t flags) {
  if ((flags & LSPCA_FORCE_SIMT) || !tc_available()) return false;
  (void)om;
  return xt == LSPCA_F32 || xt == LSPCA_BF16 || xt == LSPCA_E4M3;
}

int fit_impl(lspca_ctx* ctx, const void* X, int32_t xt, int64_t m, int64_t n, int64_t ldx, int32_t k, lspca_omega om,
             uint32_t flags, void* V, double* sigma, double* gram, int32_t* rank, void* stream, lspca_report* rep,
             bool spca) {
  if (!ctx) return LSPCA_ERR_INVALID;
  int st = check_x(X, xt, m, n, ldx);
  if (st) return st;
  if ((st = check_omega(om, xt))) return st;
  if (k < 1 || k > 256 || k > m || k > n || !V || !sigma) return LSPCA_ERR_INVALID;
  const bool want_g = (flags & LSPCA_WANT_GRAM) != 0;
  if (want_g && !gram) return LSPCA_ERR_INVALID;
  if (cudaSetDevice(ctx->device) != cudaSuccess) return LSPCA_ERR_CUDA;
  const auto t0 = std::chrono::steady_clock::now();
  cudaStream_t s = (cudaStream_t)stream;
  Launcher L{s, &ctx->launches, ctx->num_sms};
  const bool tc_s = use_tc_sketch(xt, om, flags);
  const bool tc_f = use_tc_chain(xt, flags, k);
  const size_t asz = acc_size(xt);

  // SPCA's R: CholeskyQR2 from the Gram for FP32 U on the tensor-core paths
  // (the Householder TSQR stands by, gated, for a Gram that is numerically
  // singular); the Householder TSQR alone for FP64 U and the SIMT paths
  const bool cq = spca && tc_f && xt != LSPCA_F64;
  const bool need_g = want_g || cq;

  SketchBufs sb;
  ChainBufs cb;
  SmallWs sw;
  void *U = nullptr, *small = nullptr, *qrws = nullptr;
  double *F = nullptr, *G = nullptr, *R = nullptr, *G2 = nullptr;
  float *Q1 = nullptr, *R1 = nullptr, *Rinv = nullptr, *R2 = nullptr, *cqs = nullptr;
  TcProjectWs pw2;
  TcChainWs w2;
  auto plan = [&](Plan& P) {
    U = P.take((size_t)m * k * asz);
    plan_sketch(P, sb, xt, n, k, om, tc_s, flags, m, ctx->num_sms);
    cb.f8ws = sb.f8ws;
    F = (double*)P.take((size_t)k * n * 8);
    G = (double*)P.take((size_t)k * k * 8);
    plan_chain(P, cb, xt, m, n, k, need_g, tc_f, ctx->num_sms);
    small = P.take(small_ws_bytes(k, n, nullptr));
    if (spca) {
      qrws = P.take(tsqr_ws_bytes(m, k));
      R = (double*)P.take((size_t)k * k * 8);
    }
    if (cq) {
      Q1 = (float*)P.take((size_t)m * k * 4);
      R1 = (float*)P.take((size_t)k * k * 4);
      Rinv = (float*)P.take((size_t)k * k * 4);
      R2 = (float*)P.take((size_t)k * k * 4);
      G2 = (double*)P.take((size_t)k * k * 8);
      cqs = (float*)P.take(256);  // max|Q1| twice, the failure flag
      plan_tc_project(P.base ? P.base + ((P.off + 255) & ~(size_t)255) : nullptr, pw2, LSPCA_F32, k, k);
      P.take(pw2.bytes);
      plan_tc_chain_inline(P.base ? P.base + ((P.off + 255) & ~(size_t)255) : nullptr, w2, LSPCA_F32, m, k, k, false,
                           ctx->num_sms);
      P.take(w2.bytes);
    }
  };
  Plan p0;
  plan(p0);
  if ((st = ensure_ws(ctx, p0.off + 4096, s))) return st;
  Plan p1;
  p1.base = (char*)ctx->ws;
  plan(p1);
  carve_small_ws(sw, small, k, n);

  cudaEvent_t* pe = nullptr;
  if (ctx->profiling && ctx->pcalls < (int64_t)ctx->pev.size() / 7) pe = &ctx->pev[(size_t)ctx->pcalls++ * 7];
  // report events: 0 start, 1 after pass S, 2 after pass F, 3 after QR, 4 end
  static const int rep_slot[7] = {0, -1, 1, -1, 2, 3, 4};
  Mark mark = [&](int i) {
    if (rep && rep_slot[i] >= 0) cudaEventRecord(ctx->ev[rep_slot[i]], s);
    if (pe) cudaEventRecord(pe[i], s);
  };
  cudaMemsetAsync(ctx->d_absmax, 0, 2 * sizeof(float), s);
  mark(0);
  run_sketch(ctx, L, X, xt, m, n, ldx, k, om, tc_s, sb, U, mark, spca || want_g);
  if (tc_f && !tc_s && om.kind == LSPCA_OMEGA_GAUSSIAN)
    launch_scan_x(L, U, LSPCA_F32, m, k, k, ctx->d_absmax + 1, ctx->d_status);  // max|U| for the FP16 scales
  if ((st = run_chain(ctx, L, X, xt, m, n, ldx, U, k, tc_f, cb, F, need_g ? G : nullptr, mark))) return st;
  int* cq_fail = cq ? reinterpret_cast<int*>(cqs + 2) : nullptr;
  if (cq) {
    // R1 = chol(U^T U); Q1 = U R1^-1; R2 = chol(Q1^T Q1); R = R2 R1
    cudaMemsetAsync(cqs, 0, 16, s);
    launch_chol(L, G, k, R1, cq_fail);
    launch_tri_inv(L, R1, k, Rinv, cq_fail);
    tc_project(L, U, LSPCA_F32, m, k, k, Rinv, k, pw2, Q1, ctx->d_status);
    launch_scan_x(L, Q1, LSPCA_F32, m, k, k, cqs, ctx->d_status);
    cudaMemcpyAsync(cqs + 1, cqs, sizeof(float), cudaMemcpyDeviceToDevice, s);  // X = U = Q1: one scale
    tc_chain_inline_main(L, Q1, LSPCA_F32, m, k, k, Q1, k, w2, cqs, ctx->d_status, false);
    tc_chain_reduce(L, k, k, w2, G2, nullptr);
    launch_chol(L, G2, k, R2, cq_fail);
    launch_rmul(L, R2, R1, k, R, cq_fail);
    launch_tsqr(L, U, false, m, k, qrws, R, cq_fail);  // runs only if a Cholesky broke down
    launch_trsm_rt(L, R, k, F, n, false);
  } else if (spca) {
    launch_tsqr(L, U, xt == LSPCA_F64, m, k, qrws, R);
    launch_trsm_rt(L, R, k, F, n, xt == LSPCA_F64);
  }
  mark(5);
  int32_t* rk = rank ? rank : ctx->d_rank;
  launch_decompose(L, sw, F, k, n, m, xt == LSPCA_F64, V, sigma, rk, ctx->d_status);
  if (want_g) cudaMemcpyAsync(gram, G, (size_t)k * k * 8, cudaMemcpyDeviceToDevice, s);
  mark(6);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return LSPCA_ERR_CUDA;
  if (!rep) return LSPCA_OK;

  memset(rep, 0, sizeof(*rep));
  if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return LSPCA_ERR_CUDA;
  rep->ms_sketch = ev_ms(ctx->ev[0], ctx->ev[1]);
  rep->ms_chain = ev_ms(ctx->ev[1], ctx->ev[2]);
  rep->ms_qr = ev_ms(ctx->ev[2], ctx->ev[3]);
  rep->ms_small = ev_ms(ctx->ev[3], ctx->ev[4]);
  rep->bytes_x = (double)m * n * dtype_size(xt);
  int32_t hr = 0, hst = 0, hsw = 0;
  cudaMemcpy(&hr, rk, 4, cudaMemcpyDeviceToHost);
  cudaMemcpy(&hst, ctx->d_status, 4, cudaMemcpyDeviceToHost);
  cudaMemcpy(&hsw, sw.sweeps, 4, cudaMemcpyDeviceToHost);
  cudaMemsetAsync(ctx->d_status, 0, 4, s);
  cudaStreamSynchronize(s);
  rep->rank = hr;
  rep->device_status = hst;
  rep->sweeps = hsw;
  rep->qr_path = 0;
  if (spca) {
    int32_t hf = 1;
    if (cq) cudaMemcpy(&hf, cq_fail, 4, cudaMemcpyDeviceToHost);
    rep->qr_path = hf ? 2 : 1;
  }
  rep->ms_total = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  if (hst & ST_NONFINITE) return LSPCA_ERR_NUMERIC;
  if (hst & ST_TIMEOUT) return LSPCA_ERR_TIMEOUT;
  if (hst & ST_NUMERIC) return LSPCA_ERR_NUMERIC;
  if (hr < k) return LSPCA_WARN_RANK_DEFICIENT;
  return LSPCA_OK;
}

}  // namespace

extern "C" {

int lspca_create(lspca_ctx** out, int device, size_t hbm_budget_bytes) {
  if (!out) return LSPCA_ERR_INVALID;
  *out = nullptr;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess) {
    cudaGetLastError();
    return LSPCA_ERR_CUDA;
  }
  if (device < 0 || device >= ndev) return LSPCA_ERR_INVALID;
  if (cudaSetDevice(device) != cudaSuccess) return LSPCA_ERR_CUDA;
  lspca_ctx* c = new lspca_ctx();
  c->device = device;
  cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, device);
  size_t fr = 0, tot = 0;
  cudaMemGetInfo(&fr, &tot);
  c->budget = hbm_budget_bytes ? hbm_budget_bytes : fr / 4 * 3;
  if (cudaMalloc(&c->d_status, 256) != cudaSuccess) {
    delete c;
    return LSPCA_ERR_CUDA;
  }
  cudaMemset(c->d_status, 0, 256);
  c->d_absmax = reinterpret_cast<float*>(reinterpret_cast<char*>(c->d_status) + 64);
  c->d_rank = reinterpret_cast<int32_t*>(reinterpret_cast<char*>(c->d_status) + 128);
  for (auto& e : c->ev) cudaEventCreate(&e);
  *out = c;
  return LSPCA_OK;
}

int lspca_destroy(lspca_ctx* ctx) {
  if (!ctx) return LSPCA_ERR_INVALID;
  cudaSetDevice(ctx->device);
  cudaDeviceSynchronize();
  if (ctx->ws) cudaFree(ctx->ws);
  if (ctx->aux) cudaFree(ctx->aux);
  if (ctx->d_status) cudaFree(ctx->d_status);
  for (auto& e : ctx->ev)
    if (e) cudaEventDestroy(e);
  for (int b = 0; b < 2; ++b) {
    if (ctx->copied[b]) cudaEventDestroy(ctx->copied[b]);
    if (ctx->consumed[b]) cudaEventDestroy(ctx->consumed[b]);
  }
  if (ctx->cstream) cudaStreamDestroy(ctx->cstream);
  for (auto& e : ctx->pev) cudaEventDestroy(e);
  delete ctx;
  return LSPCA_OK;
}

int lspca_fit(lspca_ctx* ctx, const void* X, int32_t xt, int64_t m, int64_t n, int64_t ldx, int32_t k, lspca_omega om,
              uint32_t flags, void* V, double* sigma, double* gram, int32_t* rank, void* stream, lspca_report* rep) {
  return fit_impl(ctx, X, xt, m, n, ldx, k, om, flags, V, sigma, gram, rank, stream, rep, false);
}

int spca_fit(lspca_ctx* ctx, const void* X, int32_t xt, int64_t m, int64_t n, int64_t ldx, int32_t k, lspca_omega om,
             uint32_t flags, void* V, double* sigma, double* gram, int32_t* rank, void* stream, lspca_report* rep) {
  return fit_impl(ctx, X, xt, m, n, ldx, k, om, flags, V, sigma, gram, rank, stream, rep, true);
}

namespace {
__global__ void rank_min_kernel(const int32_t* rl, int32_t k, int32_t* rank) { *rank = *rl < k ? *rl : k; }
}  // namespace

int lspca_fit_csr(lspca_ctx* ctx, const int64_t* row_ptr, const int32_t* col_idx, const float* val, int64_t m,
                  int64_t n, int64_t nnz, int32_t k, lspca_omega om, uint32_t flags, float* V, double* sigma,
                  int32_t* rank, void* stream, lspca_report* rep) {
  if (!ctx || !row_ptr || !V || !sigma || m < 1 || n < 1 || nnz < 0 || (nnz > 0 && (!col_idx || !val)))
    return LSPCA_ERR_INVALID;
  if (n > INT32_MAX || k < 1 || k > 256 || k > m || k > n || flags != 0) return LSPCA_ERR_INVALID;
  int st;
  if ((st = check_omega(om, LSPCA_F32))) return st;
  if (cudaSetDevice(ctx->device) != cudaSuccess) return LSPCA_ERR_CUDA;
  const auto t0 = std::chrono::steady_clock::now();
  cudaStream_t s = (cudaStream_t)stream;
  Launcher L{s, &ctx->launches, ctx->num_sms};
  float *omega = nullptr, *U = nullptr;
  double* F = nullptr;
  void *csc = nullptr, *small = nullptr;
  auto plan = [&](Plan& P) {
    omega = (float*)P.take((size_t)n * k * 4);
    U = (float*)P.take((size_t)m * k * 4);
    F = (double*)P.take((size_t)k * n * 8);
    csc = P.take(csc_ws_bytes(m, n, nnz, k));
    small = P.take(small_ws_bytes(k, n, nullptr));
  };
  Plan p0;
  plan(p0);
  if ((st = ensure_ws(ctx, p0.off + 4096, s))) return st;
  Plan p1;
  p1.base = (char*)ctx->ws;
  plan(p1);
  SmallWs sw;
  carve_small_ws(sw, small, k, n);
  if (rep) cudaEventRecord(ctx->ev[0], s);
  // U = X Omega (rows), the CSC copy, F = U^T X (columns), the k x k step
  launch_omega_dense(L, om, n, k, LSPCA_F32, omega, k, false, false);
  launch_csr_rows(L, row_ptr, col_idx, val, m, n, nnz, omega, k, U, ctx->d_status);
  if (rep) cudaEventRecord(ctx->ev[1], s);
  CscView cv;
  launch_csr_to_csc(L, row_ptr, col_idx, val, m, n, nnz, k, csc, &cv);
  launch_csc_passf(L, cv, n, nnz, U, k, F);
  if (rep) cudaEventRecord(ctx->ev[2], s);
  int32_t* rk = rank ? rank : ctx->d_rank;
  launch_decompose(L, sw, F, k, n, m, false, V, sigma, rk, ctx->d_status);
  if (rep) cudaEventRecord(ctx->ev[4], s);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return LSPCA_ERR_CUDA;
  if (!rep) return LSPCA_OK;
  memset(rep, 0, sizeof(*rep));
  if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return LSPCA_ERR_CUDA;
  rep->ms_sketch = ev_ms(ctx->ev[0], ctx->ev[1]);
  rep->ms_chain = ev_ms(ctx->ev[1], ctx->ev[2]);
  rep->ms_small = ev_ms(ctx->ev[2], ctx->ev[4]);
  rep->bytes_x = (double)nnz * 8 + (double)(m + 1) * 8;
  int32_t hr = 0, hst = 0, hsw = 0;
  cudaMemcpy(&hr, rk, 4, cudaMemcpyDeviceToHost);
  cudaMemcpy(&hst, ctx->d_status, 4, cudaMemcpyDeviceToHost);
  cudaMemcpy(&hsw, sw.sweeps, 4, cudaMemcpyDeviceToHost);
  cudaMemsetAsync(ctx->d_status, 0, 4, s);
  cudaStreamSynchronize(s);
  rep->rank = hr;
  rep->device_status = hst;
  rep->sweeps = hsw;
  rep->ms_total = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  if (hst & ST_BADINDEX) return LSPCA_ERR_INVALID;
  if (hst & ST_NONFINITE) return LSPCA_ERR_NUMERIC;
  if (hst & ST_TIMEOUT) return LSPCA_ERR_TIMEOUT;
  if (hst & ST_NUMERIC) return LSPCA_ERR_NUMERIC;
  if (hr < k) return LSPCA_WARN_RANK_DEFICIENT;
  return LSPCA_OK;
}

int lspca_project_csr(lspca_ctx* ctx, const int64_t* row_ptr, const int32_t* col_idx, const float* val, int64_t m,
                      int64_t n, int64_t nnz, const float* V, int32_t k, float* Y, void* stream) {
  if (!ctx || !row_ptr || !V || !Y || m < 1 || n < 1 || n > INT32_MAX || nnz < 0 ||
      (nnz > 0 && (!col_idx || !val)) || k < 1 || k > 256)
    return LSPCA_ERR_INVALID;
  if (cudaSetDevice(ctx->device) != cudaSuccess) return LSPCA_ERR_CUDA;
  Launcher L{(cudaStream_t)stream, &ctx->launches, ctx->num_sms};
  launch_csr_rows(L, row_ptr, col_idx, val, m, n, nnz, V, k, Y, ctx->d_status);
  return cuda_status(cudaGetLastError());
}

int lspca_fit_oversampled(lspca_ctx* ctx, const void* X, int32_t xt, int64_t m, int64_t n, int64_t ldx, int32_t k,
                          int32_t l, lspca_omega om, uint32_t flags, void* V, double* sigma, int32_t* rank,
                          void* stream, lspca_report* rep) {
  if (!ctx || !V || !sigma || k < 1 || l < k || (flags & LSPCA_WANT_GRAM)) return LSPCA_ERR_INVALID;
  if (l == k) return lspca_fit(ctx, X, xt, m, n, ldx, k, om, flags, V, sigma, nullptr, rank, stream, rep);
  if (xt < LSPCA_F64 || xt > LSPCA_E4M3 || n < 1) return LSPCA_ERR_INVALID;
  if (cudaSetDevice(ctx->device) != cudaSuccess) return LSPCA_ERR_CUDA;
  const size_t vel = xt == LSPCA_F64 ? 8 : 4;  // result type of V
  const size_t vbytes = ((size_t)n * l * vel + 255) & ~(size_t)255;
  const size_t need = vbytes + (size_t)l * 8 + 256;
  if (ctx->aux_size < need) {
    if (ctx->aux) {
      cudaDeviceSynchronize();  // the buffer may still be read by queued work
      cudaFree(ctx->aux);
      ctx->aux = nullptr;
      ctx->aux_size = 0;
    }
    if (cudaMalloc(&ctx->aux, need) != cudaSuccess) return LSPCA_ERR_NOMEM;
    ctx->aux_size = need;
  }
  char* base = (char*)ctx->aux;
  double* sl = reinterpret_cast<double*>(base + vbytes);
  int32_t* rl = reinterpret_cast<int32_t*>(base + vbytes + (((size_t)l * 8 + 255) & ~(size_t)255));
  int st = fit_impl(ctx, X, xt, m, n, ldx, l, om, flags, base, sl, nullptr, rl, stream, rep, false);
  if (st != LSPCA_OK && st != LSPCA_WARN_RANK_DEFICIENT) return st;
  cudaStream_t s = (cudaStream_t)stream;
  // top k of the l sorted singular triplets: the first k columns of every row of V
  if (cudaMemcpy2DAsync(V, (size_t)k * vel, base, (size_t)l * vel, (size_t)k * vel, (size_t)n,
                        cudaMemcpyDeviceToDevice, s) != cudaSuccess ||
      cudaMemcpyAsync(sigma, sl, (size_t)k * 8, cudaMemcpyDeviceToDevice, s) != cudaSuccess)
    return LSPCA_ERR_CUDA;
  if (rank) {
    rank_min_kernel<<<1, 1, 0, s>>>(rl, k, rank);
    ctx->launches += 1;
  }
  if (cudaGetLastError() != cudaSuccess) return LSPCA_ERR_CUDA;
  if (rep) {
    if (cudaStreamSynchronize(s) != cudaSuccess) return LSPCA_ERR_CUDA;
    if (rep->rank > k) rep->rank = k;
    if (st == LSPCA_WARN_RANK_DEFICIENT && rep->rank >= k) st = LSPCA_OK;
  }
  return st;
}

namespace {
// Algorithm 4 over a host-resident X (lspca_fit_host).  Xd (nullable): a
// device buffer of m rows x ldx that receives the slices, so X stays resident
// (no staging buffers); Yh (nullable, needs Xd): afterwards the reduction map
// of every row, slice by slice into two device staging buffers, each slice
// copied back into Yh on the copy stream while the next is projected.
int fit_host_impl(lspca_ctx* ctx, const void* Xh, int32_t xt, int64_t m, int64_t n, int64_t ldx, int32_t k,
                  lspca_omega om, uint32_t flags, int64_t slice_rows, void* V, double* sigma, int32_t* rank,
                  void* stream, lspca_report* rep, void* Xd, float* Yh) {
  if (!ctx || !Xh || !V || !sigma) return LSPCA_ERR_INVALID;
  if (Yh && !Xd) return LSPCA_ERR_INVALID;
  if (Xd && ((uintptr_t)Xd & 15u)) return LSPCA_ERR_INVALID;
  if (xt != LSPCA_F32 && xt != LSPCA_BF16 && xt != LSPCA_E4M3) return LSPCA_ERR_INVALID;
  if (m < 1 || n < 1 || ldx < n || (ldx * (int64_t)dtype_size(xt)) % 16 != 0) return LSPCA_ERR_INVALID;
  int st;
  if ((st = check_omega(om, xt))) return st;
  if (k < 1 || k > 256 || k > m || k > n || (k % 4) != 0 || slice_rows < 0) return LSPCA_ERR_INVALID;
  if (flags & (LSPCA_WANT_GRAM | LSPCA_FORCE_SIMT)) return LSPCA_ERR_INVALID;
  if (cudaSetDevice(ctx->device) != cudaSuccess) return LSPCA_ERR_CUDA;
  if (!tc_available()) return LSPCA_ERR_INVALID;
  const auto t0 = std::chrono::steady_clock::now();
  cudaStream_t s = (cudaStream_t)stream;
  Launcher L{s, &ctx->launches, ctx->num_sms};
  const int64_t row_bytes = ldx * (int64_t)dtype_size(xt);
  if (slice_rows == 0) slice_rows = ((int64_t)256 << 20) / row_bytes;  // ~256 MB slices
  slice_rows = (slice_rows + 127) / 128 * 128;
  if (slice_rows < 128) slice_rows = 128;
  if (slice_rows > m) slice_rows = m;
  const int64_t nslices = (m + slice_rows - 1) / slice_rows;
  const bool exact = om.kind == LSPCA_OMEGA_VERY_SPARSE;

  // projection slices: about 128 MB of Y each, whole 128-row tiles
  int64_t proj_rows = (((int64_t)128 << 20) / ((int64_t)k * 4) + 127) / 128 * 128;
  if (proj_rows > m) proj_rows = (m + 127) / 128 * 128;
  void *stage[2] = {nullptr, nullptr}, *U = nullptr, *omega_d = nullptr, *tiles = nullptr, *small = nullptr;
  float* scal = nullptr;
  float* ystage[2] = {nullptr, nullptr};
  double* Facc = nullptr;
  char* chain_base = nullptr;
  TcChainWs cw_max;
  TcProjectWs pw;
  auto plan = [&](Plan& P) {
    if (!Xd)
      for (auto& b : stage) b = P.take((size_t)slice_rows * (size_t)row_bytes);
    if (Yh) {
      for (auto& b : ystage) b = (float*)P.take((size_t)proj_rows * k * 4);
      char* base = P.base ? P.base + ((P.off + 255) & ~(size_t)255) : nullptr;
      plan_tc_project(base, pw, xt, n, k);
      P.take(pw.bytes);
    }
    U = P.take((size_t)slice_rows * k * 4);
    omega_d = P.take((size_t)n * k * 4);
    tiles = P.take(tc_tile_v_bytes(n, k));
    scal = (float*)P.take(256);
    Facc = (double*)P.take((size_t)k * n * 8);
    small = P.take(small_ws_bytes(k, n, nullptr));
    plan_tc_chain(nullptr, cw_max, xt, slice_rows, n, k, false, ctx->num_sms);
    chain_base = (char*)P.take(cw_max.bytes);
  };
  Plan p0;
  plan(p0);
  if ((st = ensure_ws(ctx, p0.off + 4096, s))) return st;
  Plan p1;
  p1.base = (char*)ctx->ws;
  plan(p1);
  SmallWs sw;
  carve_small_ws(sw, small, k, n);
  if (!ctx->cstream) {
    if (cudaStreamCreateWithFlags(&ctx->cstream, cudaStreamNonBlocking) != cudaSuccess) return LSPCA_ERR_CUDA;
    for (int b = 0; b < 2; ++b) {
      if (cudaEventCreateWithFlags(&ctx->copied[b], cudaEventDisableTiming) != cudaSuccess ||
          cudaEventCreateWithFlags(&ctx->consumed[b], cudaEventDisableTiming) != cudaSuccess)
        return LSPCA_ERR_CUDA;
    }
  }
  // Omega once per fit, tiled for the reduction-map kernel
  if (rep) cudaEventRecord(ctx->ev[0], s);
  launch_omega_dense(L, om, n, k, LSPCA_F32, omega_d, k, false, xt == LSPCA_BF16);
  tc_tile_v(L, xt, (const float*)omega_d, n, k, tiles, scal, ctx->d_status, exact);
  // the copy stream starts after the work already queued on the caller's stream
  // (the staging buffers may still be read by a previous call)
  cudaEventRecord(ctx->consumed[0], s);
  cudaStreamWaitEvent(ctx->cstream, ctx->consumed[0], 0);
  for (int64_t si = 0; si < nslices; ++si) {
    const int b = (int)(si & 1);
    const int64_t r0 = si * slice_rows;
    const int64_t rows = (r0 + slice_rows <= m) ? slice_rows : m - r0;
    // Algorithm 4: copy slice si while the previous slice is computed (into
    // the resident X, or into the staging buffer the slice before last freed)
    void* xs = Xd ? (void*)((char*)Xd + r0 * row_bytes) : stage[b];
    if (!Xd && si >= 2) cudaStreamWaitEvent(ctx->cstream, ctx->consumed[b], 0);
    if (cudaMemcpyAsync(xs, (const char*)Xh + r0 * row_bytes, (size_t)(rows * row_bytes), cudaMemcpyHostToDevice,
                        ctx->cstream) != cudaSuccess)
      return LSPCA_ERR_CUDA;
    cudaEventRecord(ctx->copied[b], ctx->cstream);
    cudaStreamWaitEvent(s, ctx->copied[b], 0);
    // U_s = X_s Omega (max|X_s|, NaN / Inf, max|U_s| taken on the way); F += U_s^T X_s
    cudaMemsetAsync(ctx->d_absmax, 0, 2 * sizeof(float), s);
    tc_project_pretiled(L, xs, xt, rows, n, ldx, tiles, scal + 1, k, (float*)U, ctx->d_status, exact,
                        ctx->d_absmax, ctx->d_absmax + 1);
    TcChainWs cw;
    plan_tc_chain(chain_base, cw, xt, rows, n, k, false, ctx->num_sms);
    if (!tc_chain_main(L, xs, xt, rows, n, ldx, (const float*)U, k, cw, ctx->d_absmax, ctx->d_status, false))
      return LSPCA_ERR_CUDA;
    tc_chain_reduce(L, n, k, cw, Facc, nullptr, si > 0);
    cudaEventRecord(ctx->consumed[b], s);
  }
  if (rep) cudaEventRecord(ctx->ev[2], s);
  int32_t* rk = rank ? rank : ctx->d_rank;
  launch_decompose(L, sw, Facc, k, n, m, false, V, sigma, rk, ctx->d_status);
  if (rep) cudaEventRecord(ctx->ev[4], s);
  if (Yh) {
    // Y = X V slice by slice; slice q is copied back on the copy stream while
    // slice q + 1 is projected (two staging buffers)
    const bool pre = tc_xproj_tile_v(L, xt, (const float*)V, n, k, pw, ctx->d_status);
    const int64_t npslices = (m + proj_rows - 1) / proj_rows;
    for (int64_t q = 0; q < npslices; ++q) {
      const int b = (int)(q & 1);
      const int64_t r0 = q * proj_rows;
      const int64_t rows = (r0 + proj_rows <= m) ? proj_rows : m - r0;
      const void* xs = (const char*)Xd + r0 * row_bytes;
      if (q >= 2) cudaStreamWaitEvent(s, ctx->consumed[b], 0);  // staging buffer b copied out
      if (!(pre && tc_xproj(L, xs, xt, rows, n, ldx, pw.vhi, (const float*)pw.vlo + 1, k, false, ystage[b],
                            ctx->d_status, nullptr, false))) {
        if (pre) return LSPCA_ERR_CUDA;
        tc_project(L, xs, xt, rows, n, ldx, (const float*)V, k, pw, ystage[b], ctx->d_status);
      }
      cudaEventRecord(ctx->copied[b], s);
      cudaStreamWaitEvent(ctx->cstream, ctx->copied[b], 0);
      if (cudaMemcpyAsync(Yh + r0 * k, ystage[b], (size_t)rows * k * 4, cudaMemcpyDeviceToHost, ctx->cstream) !=
          cudaSuccess)
        return LSPCA_ERR_CUDA;
      cudaEventRecord(ctx->consumed[b], ctx->cstream);
    }
    // the caller's stream completes only after the last copy of Y
    cudaEventRecord(ctx->consumed[0], ctx->cstream);
    cudaStreamWaitEvent(s, ctx->consumed[0], 0);
    if (rep) cudaEventRecord(ctx->ev[5], s);
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return LSPCA_ERR_CUDA;
  if (!rep) return LSPCA_OK;
  memset(rep, 0, sizeof(*rep));
  if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return LSPCA_ERR_CUDA;
  rep->ms_chain = ev_ms(ctx->ev[0], ctx->ev[2]);  // copies, sketches and pass F of all slices
  rep->ms_small = ev_ms(ctx->ev[2], ctx->ev[4]);
  if (Yh) rep->ms_qr = ev_ms(ctx->ev[4], ctx->ev[5]);  // the reduction map and the copies of Y
  rep->bytes_x = (double)m * n * dtype_size(xt);
  int32_t hr = 0, hst = 0, hsw = 0;
  cudaMemcpy(&hr, rk, 4, cudaMemcpyDeviceToHost);
  cudaMemcpy(&hst, ctx->d_status, 4, cudaMemcpyDeviceToHost);
  cudaMemcpy(&hsw, sw.sweeps, 4, cudaMemcpyDeviceToHost);
  cudaMemsetAsync(ctx->d_status, 0, 4, s);
  cudaStreamSynchronize(s);
  rep->rank = hr;
  rep->device_status = hst;
  rep->sweeps = hsw;
  rep->ms_total = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  if (hst & ST_NONFINITE) return LSPCA_ERR_NUMERIC;
  if (hst & ST_TIMEOUT) return LSPCA_ERR_TIMEOUT;
  if (hst & ST_NUMERIC) return LSPCA_ERR_NUMERIC;
  if (hr < k) return LSPCA_WARN_RANK_DEFICIENT;
  return LSPCA_OK;
}
}  // namespace

int lspca_fit_host(lspca_ctx* ctx, const void* Xh, int32_t xt, int64_t m, int64_t n, int64_t ldx, int32_t k,
                   lspca_omega om, uint32_t flags, int64_t slice_rows, void* V, double* sigma, int32_t* rank,
                   void* stream, lspca_report* rep) {
  return fit_host_impl(ctx, Xh, xt, m, n, ldx, k, om, flags, slice_rows, V, sigma, rank, stream, rep, nullptr,
                       nullptr);
}

int lspca_fit_project_host(lspca_ctx* ctx, const void* Xh, int32_t xt, int64_t m, int64_t n, int64_t ldx, int32_t k,
                           lspca_omega om, uint32_t flags, int64_t slice_rows, void* Xd, void* V, double* sigma,
                           int32_t* rank, float* Yh, void* stream, lspca_report* rep) {
  if (!Xd || !Yh) return LSPCA_ERR_INVALID;
  return fit_host_impl(ctx, Xh, xt, m, n, ldx, k, om, flags, slice_rows, V, sigma, rank, stream, rep, Xd, Yh);
}

int lspca_project(lspca_ctx* ctx, const void* X, int32_t xt, int64_t m, int64_t n, int64_t ldx, const void* V,
                  int32_t k, void* Y, void* stream) {
  if (!ctx) return LSPCA_ERR_INVALID;
  int st = check_x(X, xt, m, n, ldx);
  if (st) return st;
  if (!V || !Y || k < 1 || k > 256) return LSPCA_ERR_INVALID;
  if (cudaSetDevice(ctx->device) != cudaSuccess) return LSPCA_ERR_CUDA;
  cudaStream_t s = (cudaStream_t)stream;
  Launcher L{s, &ctx->launches, ctx->num_sms};
  if (xt != LSPCA_F64 && tc_available() && aligned16(V)) {
    TcProjectWs pw;
    plan_tc_project(nullptr, pw, xt, n, k);
    if ((st = ensure_ws(ctx, pw.bytes + 4096, s))) return st;
    plan_tc_project((char*)ctx->ws, pw, xt, n, k);
    tc_project(L, X, xt, m, n, ldx, (const float*)V, k, pw, (float*)Y, ctx->d_status);
  } else {
    launch_gemm_simt(L, m, k, n, X, xt, ldx, false, V, acc_dt(xt), k, false, Y, xt == LSPCA_F64, k, 0, 1,
                     xt == LSPCA_F64, false);
  }
  return cuda_status(cudaGetLastError());
}

int lspca_omega_materialize(lspca_ctx* ctx, lspca_omega om, int64_t n, int32_t k, int32_t t, void* out,
                            void* stream) {
  if (!ctx || !out || n < 1 || k < 1) return LSPCA_ERR_INVALID;
  if (t != LSPCA_F64 && t != LSPCA_F32 && t != LSPCA_BF16) return LSPCA_ERR_INVALID;
  if (om.kind != LSPCA_OMEGA_GAUSSIAN && om.kind != LSPCA_OMEGA_VERY_SPARSE) return LSPCA_ERR_INVALID;
  if (om.kind == LSPCA_OMEGA_VERY_SPARSE && om.p == 0) return LSPCA_ERR_INVALID;
  if (cudaSetDevice(ctx->device) != cudaSuccess) return LSPCA_ERR_CUDA;
  Launcher L{(cudaStream_t)stream, &ctx->launches, ctx->num_sms};
  launch_omega_dense(L, om, n, k, t, out, k, false, t == LSPCA_BF16);
  return cuda_status(cudaGetLastError());
}

int lspca_sketch(lspca_ctx* ctx, const void* X, int32_t xt, int64_t m, int64_t n, int64_t ldx, int32_t k,
                 lspca_omega om, uint32_t flags, void* U, void* stream) {
  if (!ctx) return LSPCA_ERR_INVALID;
  int st = check_x(X, xt, m, n, ldx);
  if (st) return st;
  if ((st = check_omega(om, xt))) return st;
  if (!U || k < 1 || k > 256) return LSPCA_ERR_INVALID;
  if (cudaSetDevice(ctx->device) != cudaSuccess) return LSPCA_ERR_CUDA;
  cudaStream_t s = (cudaStream_t)stream;
  Launcher L{s, &ctx->launches, ctx->num_sms};
  const bool tc = use_tc_sketch(xt, om, flags);
  SketchBufs sb;
  Plan p0;
  plan_sketch(p0, sb, xt, n, k, om, tc, flags, m, ctx->num_sms);
  if ((st = ensure_ws(ctx, p0.off + 4096, s))) return st;
  Plan p1;
  p1.base = (char*)ctx->ws;
  plan_sketch(p1, sb, xt, n, k, om, tc, flags, m, ctx->num_sms);
  cudaMemsetAsync(ctx->d_absmax, 0, 2 * sizeof(float), s);
  run_sketch(ctx, L, X, xt, m, n, ldx, k, om, tc, sb, U, [](int) {});
  return cuda_status(cudaGetLastError());
}

int lspca_sum_partials(lspca_ctx* ctx, const double* parts, int32_t nparts, int64_t count, double* out,
                       void* stream) {
  if (!ctx || !parts || !out || nparts < 1 || count < 0) return LSPCA_ERR_INVALID;
  if (count == 0) return LSPCA_OK;
  if (cudaSetDevice(ctx->device) != cudaSuccess) return LSPCA_ERR_CUDA;
  Launcher L{(cudaStream_t)stream, &ctx->launches, ctx->num_sms};
  launch_reduce_splits(L, parts, nparts, count, count, out);
  return cuda_status(cudaGetLastError());
}

int lspca_chain(lspca_ctx* ctx, const void* X, int32_t xt, int64_t m, int64_t n, int64_t ldx, const void* U, int32_t k,
                uint32_t flags, double* F, double* G, void* stream) {
  if (!ctx) return LSPCA_ERR_INVALID;
  int st = check_x(X, xt, m, n, ldx);
  if (st) return st;
  if (!U || !F || k < 1 || k > 256) return LSPCA_ERR_INVALID;
  if (cudaSetDevice(ctx->device) != cudaSuccess) return LSPCA_ERR_CUDA;
  cudaStream_t s = (cudaStream_t)stream;
  Launcher L{s, &ctx->launches, ctx->num_sms};
  const bool tc = use_tc_chain(xt, flags, k) && aligned16(U);
  const bool f8 = tc && use_f8(xt, flags);
  ChainBufs cb;
  auto plan = [&](Plan& P) {
    plan_chain(P, cb, xt, m, n, k, G != nullptr, tc, ctx->num_sms);
    if (f8) cb.f8ws = P.take(f8_ws_bytes(m, n, k, ctx->num_sms));
  };
  Plan p0;
  plan(p0);
  if ((st = ensure_ws(ctx, p0.off + 4096, s))) return st;
  Plan p1;
  p1.base = (char*)ctx->ws;
  plan(p1);
  // the FP8 pass F reads U as E4M3 bytes (exact, or flagged and left to the BF16 pass F)
  if (f8) launch_f8_u8(L, (const float*)U, m, k, cb.f8ws, n);
  if (tc) {
    // the split-FP16 path scales by powers of two derived from max|X| and max|U|
    cudaMemsetAsync(ctx->d_absmax, 0, 2 * sizeof(float), s);
    launch_scan_x(L, X, xt, m, n, ldx, ctx->d_absmax, ctx->d_status);
    launch_scan_x(L, U, LSPCA_F32, m, k, k, ctx->d_absmax + 1, ctx->d_status);
  }
  if ((st = run_chain(ctx, L, X, xt, m, n, ldx, U, k, tc, cb, F, G, [](int) {}))) return st;
  return cuda_status(cudaGetLastError());
}

int lspca_decompose(lspca_ctx* ctx, const double* F, int32_t k, int64_t n, int64_t m, int32_t vt, void* V,
                    double* sigma, int32_t* rank, void* stream) {
  if (!ctx || !F || !V || k < 1 || k > 256 || n < k || m < 1) return LSPCA_ERR_INVALID;
  if (vt != LSPCA_F64 && vt != LSPCA_F32) return LSPCA_ERR_INVALID;
  if (cudaSetDevice(ctx->device) != cudaSuccess) return LSPCA_ERR_CUDA;
  cudaStream_t s = (cudaStream_t)stream;
  Launcher L{s, &ctx->launches, ctx->num_sms};
  int st;
  const size_t bytes = small_ws_bytes(k, n, nullptr);
  if ((st = ensure_ws(ctx, bytes + 4096, s))) return st;
  SmallWs sw;
  carve_small_ws(sw, ctx->ws, k, n);
  launch_decompose(L, sw, F, k, n, m, vt == LSPCA_F64, V, sigma, rank ? rank : ctx->d_rank, ctx->d_status);
  return cuda_status(cudaGetLastError());
}

int lspca_wait_probe(lspca_ctx* ctx, int64_t limit_ns, int64_t* waited_ns, void* stream) {
  if (!ctx || limit_ns < 1000 || limit_ns > 2000000000ll) return LSPCA_ERR_INVALID;
  if (cudaSetDevice(ctx->device) != cudaSuccess) return LSPCA_ERR_CUDA;
  Launcher L{(cudaStream_t)stream, &ctx->launches, ctx->num_sms};
  launch_wait_probe(L, (uint64_t)limit_ns, ctx->d_status, waited_ns);
  return cuda_status(cudaGetLastError());
}

int lspca_sync_status(lspca_ctx* ctx, void* stream) {
  if (!ctx) return LSPCA_ERR_INVALID;
  if (cudaSetDevice(ctx->device) != cudaSuccess) return LSPCA_ERR_CUDA;
  cudaStream_t s = (cudaStream_t)stream;
  if (cudaStreamSynchronize(s) != cudaSuccess) return LSPCA_ERR_CUDA;
  int32_t h = 0;
  if (cudaMemcpy(&h, ctx->d_status, 4, cudaMemcpyDeviceToHost) != cudaSuccess) return LSPCA_ERR_CUDA;
  cudaMemset(ctx->d_status, 0, 4);
  if (h & ST_BADINDEX) return LSPCA_ERR_INVALID;
  if (h & ST_NONFINITE) return LSPCA_ERR_NUMERIC;
  if (h & ST_TIMEOUT) return LSPCA_ERR_TIMEOUT;
  if (h & ST_NUMERIC) return LSPCA_ERR_NUMERIC;
  return LSPCA_OK;
}

const char* lspca_strerror(int status) {
  switch (status) {
    case LSPCA_OK: return "ok";
    case LSPCA_ERR_INVALID: return "invalid argument";
    case LSPCA_ERR_NOMEM: return "workspace exceeds the context's HBM budget";
    case LSPCA_WARN_RANK_DEFICIENT: return "rank deficient (rank < k)";
    case LSPCA_ERR_NUMERIC: return "non-finite input or numeric failure";
    case LSPCA_ERR_TIMEOUT: return "a bounded wait gave up";
    case LSPCA_ERR_CUDA: return "CUDA error";
    case LSPCA_ERR_BUSY: return "busy: no free slot or over budget";
    default: return "unknown status";
  }
}

int64_t lspca_launch_count(lspca_ctx* ctx) { return ctx ? ctx->launches : 0; }

int lspca_profile(lspca_ctx* ctx, int enable) {
  if (!ctx) return LSPCA_ERR_INVALID;
  if (cudaSetDevice(ctx->device) != cudaSuccess) return LSPCA_ERR_CUDA;
  cudaDeviceSynchronize();
  for (auto& e : ctx->pev) cudaEventDestroy(e);
  ctx->pev.clear();
  ctx->pcalls = 0;
  ctx->profiling = enable != 0;
  if (enable) {
    ctx->pev.resize(4096 * 7);
    for (auto& e : ctx->pev)
      if (cudaEventCreate(&e) != cudaSuccess) return LSPCA_ERR_CUDA;
  }
  return LSPCA_OK;
}

int lspca_profile_read(lspca_ctx* ctx, double* ms7, int64_t* calls) {
  if (!ctx || !ms7) return LSPCA_ERR_INVALID;
  if (cudaSetDevice(ctx->device) != cudaSuccess) return LSPCA_ERR_CUDA;
  if (cudaDeviceSynchronize() != cudaSuccess) return LSPCA_ERR_CUDA;
  for (int i = 0; i < 7; ++i) ms7[i] = 0.0;
  for (int64_t c = 0; c < ctx->pcalls; ++c) {
    cudaEvent_t* e = &ctx->pev[(size_t)c * 7];
    for (int i = 0; i < 6; ++i) ms7[i] += ev_ms(e[i], e[i + 1]);
    ms7[6] += ev_ms(e[0], e[6]);
  }
  if (calls) *calls = ctx->pcalls;
  return LSPCA_OK;
}

}  // extern "C"
