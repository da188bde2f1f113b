// Serving runtime: continuous batching of reduction-map (projection) requests
// and Lazy SPCA fit requests on one GPU.
//
// * Requests queue on submit (their X, Y, V buffers are device memory owned by
//   the caller).  Each lspca_srv_step admits queued requests in FIFO order while
//   a slot is free and, for fits, while the request's workspace fits the
//   server's HBM arena (first-fit allocation); a request that does not fit waits
//   at the head of the queue until memory frees up.
// * Projections: every running request contributes its 128-row tiles; the tiles
//   of all requests with the same X type and padded k form one table, and one
//   persistent launch of the tensor-core reduction-map kernel walks the table
//   (requests of uneven row counts share the launch).  The table copy and the
//   launch are captured once per group as a CUDA graph and replayed every step
//   (two graphs per group alternate over two pinned host tables).
// * Fits follow Algorithm 4: every step advances each running fit by one slice
//   of rows (sketch of the slice, pass F of the slice, F += F_slice in FP64);
//   after the last slice the k x k step produces V and sigma.  Slices are fixed
//   per request, so a fit's arithmetic does not depend on what else runs.
// * Projections run on a high-priority stream and fit slices on a low-priority
//   one, so a projection waits for at most the fit kernel that occupies the
//   SMs when it arrives, not for the fit slices queued behind it.
// * A batch records one event per stream; the requests it completes are done
//   when that event has completed (lspca_srv_poll / lspca_srv_wait with a
//   bounded wait).
#include <algorithm>
#include <chrono>
#include <cstring>
#include <deque>
#include <map>
#include <thread>
#include <unordered_map>
#include <vector>

#include "common.cuh"
#include "kernels.h"
#include "tc.h"

namespace lspca {
namespace {

constexpr int kGroups = 12;        // 3 X types x 4 padded-k classes
constexpr int kMaxTiles = 2048;    // tiles per group per step
constexpr int64_t kFitSlice = 65536;

int group_of(int xt, int k) {
  const int x = xt == LSPCA_F32 ? 0 : (xt == LSPCA_BF16 ? 1 : 2);
  return x * 4 + ((k + 63) / 64 - 1);
}

__global__ void add_f64_kernel(double* __restrict__ acc, const double* __restrict__ x, int64_t count) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < count; e += (int64_t)gridDim.x * blockDim.x)
    acc[e] += x[e];
}

struct SrvV {
  const float* V = nullptr;
  int64_t n = 0;
  int k = 0;
  size_t tiles_off[3] = {0, 0, 0};  // arena offsets of the tiles per X type
  bool ready[3] = {false, false, false};
};

enum { REQ_QUEUED = 0, REQ_RUNNING = 1, REQ_DONE = 2, REQ_FAILED = 3 };
enum { KIND_PROJECT = 0, KIND_FIT = 1 };

struct Req {
  int64_t id = 0;
  int kind = 0;
  int state = REQ_QUEUED;
  const void* X = nullptr;
  int xt = 0;
  int64_t rows = 0, ldx = 0, n = 0;
  int k = 0;
  int64_t next = 0;
  bool finishing = false;
  cudaEvent_t ev = nullptr;
  // projection
  int v = -1;
  float* Y = nullptr;
  // fit
  lspca_omega om{};
  float* Vout = nullptr;
  double* sigma = nullptr;
  size_t ws_off = 0, ws_bytes = 0;
  bool prepared = false;
};

}  // namespace
}  // namespace lspca

using namespace lspca;

struct lspca_srv {
  int device = 0;
  int num_sms = 0;
  cudaStream_t stream = nullptr;   // fits (low priority)
  cudaStream_t pstream = nullptr;  // projections (high priority)
  char* arena = nullptr;
  size_t arena_size = 0;
  std::map<size_t, size_t> free_blocks;  // offset -> size
  int max_inflight = 64;
  int inflight = 0;
  std::vector<SrvV> vs;
  std::deque<int64_t> queue;
  std::vector<int64_t> running;  // admission order
  std::unordered_map<int64_t, Req> reqs;
  int64_t next_id = 1;
  // projection tables: [group][buffer]
  TcProjUnit* h_units[kGroups][2] = {};
  int* h_count[kGroups][2] = {};
  TcProjUnit* d_units[kGroups] = {};
  int* d_count[kGroups] = {};
  cudaGraphExec_t gexec[kGroups][2] = {};
  cudaEvent_t buf_ev[kGroups][2] = {};
  int flip[kGroups] = {};
  bool warmed[kGroups] = {};
  int* d_status = nullptr;
  int64_t launches = 0;
  std::vector<cudaEvent_t> ev_pool;
};

namespace {

bool arena_alloc(lspca_srv* s, size_t bytes, size_t* off) {
  bytes = (bytes + 255) & ~(size_t)255;
  for (auto it = s->free_blocks.begin(); it != s->free_blocks.end(); ++it) {
    if (it->second >= bytes) {
      *off = it->first;
      const size_t rest = it->second - bytes, noff = it->first + bytes;
      s->free_blocks.erase(it);
      if (rest) s->free_blocks[noff] = rest;
      return true;
    }
  }
  return false;
}

void arena_free(lspca_srv* s, size_t off, size_t bytes) {
  bytes = (bytes + 255) & ~(size_t)255;
  auto it = s->free_blocks.emplace(off, bytes).first;
  auto nx = std::next(it);
  if (nx != s->free_blocks.end() && it->first + it->second == nx->first) {
    it->second += nx->second;
    s->free_blocks.erase(nx);
  }
  if (it != s->free_blocks.begin()) {
    auto pv = std::prev(it);
    if (pv->first + pv->second == it->first) {
      pv->second += it->second;
      s->free_blocks.erase(it);
    }
  }
}

cudaEvent_t take_event(lspca_srv* s) {
  if (!s->ev_pool.empty()) {
    cudaEvent_t e = s->ev_pool.back();
    s->ev_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreateWithFlags(&e, cudaEventDisableTiming);
  return e;
}

// ---- fit workspace layout (one arena block per fit) -------------------------
struct FitLayout {
  size_t U = 0, counts = 0, colp = 0, ent = 0, off = 0, omega = 0, tiles = 0, scal = 0, chain = 0, fslice = 0,
         facc = 0, small = 0, misc = 0, total = 0;
  TcChainWs cw;
};

bool fit_tc_sketch(const Req& r) {
  return (r.om.kind == LSPCA_OMEGA_GAUSSIAN && (r.xt == LSPCA_F32 || r.xt == LSPCA_BF16)) || r.xt == LSPCA_E4M3;
}

FitLayout fit_layout(const Req& r, int num_sms) {
  FitLayout L;
  size_t o = 0;
  auto take = [&](size_t b) {
    o = (o + 255) & ~(size_t)255;
    const size_t at = o;
    o += b;
    return at;
  };
  const int64_t slice = r.rows < kFitSlice ? r.rows : kFitSlice;
  L.U = take((size_t)slice * r.k * 4);
  if (fit_tc_sketch(r)) {
    L.omega = take((size_t)r.n * r.k * 4);
    L.tiles = take(tc_tile_v_bytes(r.n, r.k));
    L.scal = take(256);
  } else {
    L.counts = take((size_t)r.k * 4);
    L.colp = take((size_t)(r.k + 1) * 4);
    L.ent = take((size_t)r.n * r.k * 4);
    L.off = take(sketch_off_bytes(r.n, r.k));
  }
  plan_tc_chain(nullptr, L.cw, r.xt, slice, r.n, r.k, false, num_sms);
  L.chain = take(L.cw.bytes);
  L.fslice = take((size_t)r.k * r.n * 8);
  L.facc = take((size_t)r.k * r.n * 8);
  L.small = take(small_ws_bytes(r.k, r.n, nullptr));
  L.misc = take(256);  // absmax[2], status, rank
  L.total = o + 256;
  return L;
}

void fit_prepare(lspca_srv* s, Req& r, Launcher& L) {
  const FitLayout F = fit_layout(r, s->num_sms);
  char* b = s->arena + r.ws_off;
  if (fit_tc_sketch(r)) {
    launch_omega_dense(L, r.om, r.n, r.k, LSPCA_F32, b + F.omega, r.k, false, r.xt == LSPCA_BF16);
    tc_tile_v(L, r.xt, (const float*)(b + F.omega), r.n, r.k, b + F.tiles, (float*)(b + F.scal), s->d_status);
  } else {
    launch_omega_csc(L, r.om, r.n, r.k, (int32_t*)(b + F.counts), (int32_t*)(b + F.colp), (int32_t*)(b + F.ent));
  }
  cudaMemsetAsync(b + F.facc, 0, (size_t)r.k * r.n * 8, L.stream);
  r.prepared = true;
}

bool fit_slice(lspca_srv* s, Req& r, Launcher& L) {
  FitLayout F = fit_layout(r, s->num_sms);
  char* b = s->arena + r.ws_off;
  const int64_t r0 = r.next;
  int64_t rows = r.rows - r0;
  if (rows > kFitSlice) rows = kFitSlice;
  const char* Xs = (const char*)r.X + r0 * r.ldx * (int64_t)dtype_size(r.xt);
  float* U = (float*)(b + F.U);
  float* absmax = (float*)(b + F.misc);
  cudaMemsetAsync(absmax, 0, 8, L.stream);
  if (fit_tc_sketch(r)) {
    // U_s = X_s Omega on the reduction-map kernel with the request's pre-tiled
    // Omega; the kernel takes max|X_s| (NaN / Inf detection) and max|U_s|
    tc_project_pretiled(L, Xs, r.xt, rows, r.n, r.ldx, b + F.tiles, (const float*)(b + F.scal) + 1, r.k, U,
                        s->d_status, r.om.kind == LSPCA_OMEGA_VERY_SPARSE, absmax, absmax + 1);
  } else {
    launch_sketch_sparse(L, Xs, r.xt, rows, r.n, r.ldx, r.k, (const int32_t*)(b + F.colp), (const int32_t*)(b + F.ent),
                         (int32_t*)(b + F.off), U, r.k, absmax, s->d_status);
  }
  // pass F of the slice; the chunking depends only on the slice size
  TcChainWs cw;
  plan_tc_chain(b + F.chain, cw, r.xt, rows, r.n, r.k, false, s->num_sms);
  if (!tc_chain_main(L, Xs, r.xt, rows, r.n, r.ldx, U, r.k, cw, absmax, s->d_status, false)) return false;
  tc_chain_reduce(L, r.n, r.k, cw, (double*)(b + F.fslice), nullptr);
  const int64_t cnt = (int64_t)r.k * r.n;
  add_f64_kernel<<<(int)((cnt + 255) / 256 < 4 * s->num_sms ? (cnt + 255) / 256 : 4 * s->num_sms), 256, 0,
                   L.stream>>>((double*)(b + F.facc), (const double*)(b + F.fslice), cnt);
  L.count(1);
  r.next += rows;
  if (r.next >= r.rows) {
    SmallWs sw;
    carve_small_ws(sw, b + F.small, r.k, r.n);
    launch_decompose(L, sw, (const double*)(b + F.facc), r.k, r.n, r.rows, false, r.Vout, r.sigma,
                     (int32_t*)(b + F.misc + 64), s->d_status);
    r.finishing = true;
  }
  return true;
}

bool tc_ok(int xt, int k) { return xt != LSPCA_F64 && k >= 4 && k <= 256 && (k % 4) == 0 && tc_available(); }

// Retire requests whose completion event has fired: free fit workspaces and slots.
void retire(lspca_srv* s) {
  std::vector<int64_t> keep;
  for (int64_t id : s->running) {
    Req& r = s->reqs[id];
    if (r.finishing && r.ev && cudaEventQuery(r.ev) == cudaSuccess) {
      r.state = REQ_DONE;
      if (r.kind == KIND_FIT && r.ws_bytes) arena_free(s, r.ws_off, r.ws_bytes);
      s->inflight--;
      s->ev_pool.push_back(r.ev);
      r.ev = nullptr;
      continue;
    }
    keep.push_back(id);
  }
  s->running.swap(keep);
}

}  // namespace

extern "C" {

int lspca_srv_create(lspca_srv** out, int device, size_t hbm_budget_bytes, int32_t max_inflight) {
  if (!out || max_inflight < 1) return LSPCA_ERR_INVALID;
  *out = nullptr;
  if (cudaSetDevice(device) != cudaSuccess) return LSPCA_ERR_CUDA;
  lspca_srv* s = new lspca_srv();
  s->device = device;
  s->max_inflight = max_inflight;
  cudaDeviceGetAttribute(&s->num_sms, cudaDevAttrMultiProcessorCount, device);
  int least = 0, greatest = 0;
  cudaDeviceGetStreamPriorityRange(&least, &greatest);
  if (cudaStreamCreateWithPriority(&s->stream, cudaStreamNonBlocking, least) != cudaSuccess) {
    delete s;
    return LSPCA_ERR_CUDA;
  }
  if (cudaStreamCreateWithPriority(&s->pstream, cudaStreamNonBlocking, greatest) != cudaSuccess) {
    cudaStreamDestroy(s->stream);
    delete s;
    return LSPCA_ERR_CUDA;
  }
  if (!hbm_budget_bytes) hbm_budget_bytes = (size_t)4 << 30;
  if (cudaMalloc(&s->arena, hbm_budget_bytes) != cudaSuccess) {
    cudaGetLastError();
    cudaStreamDestroy(s->stream);
    cudaStreamDestroy(s->pstream);
    delete s;
    return LSPCA_ERR_NOMEM;
  }
  s->arena_size = hbm_budget_bytes;
  s->free_blocks[0] = hbm_budget_bytes;
  cudaMalloc(&s->d_status, 256);
  cudaMemset(s->d_status, 0, 256);
  for (int g = 0; g < kGroups; ++g) {
    cudaMalloc(&s->d_units[g], sizeof(TcProjUnit) * kMaxTiles);
    cudaMalloc(&s->d_count[g], 64);
    for (int b = 0; b < 2; ++b) {
      cudaHostAlloc(&s->h_units[g][b], sizeof(TcProjUnit) * kMaxTiles, cudaHostAllocDefault);
      cudaHostAlloc(&s->h_count[g][b], 64, cudaHostAllocDefault);
      cudaEventCreateWithFlags(&s->buf_ev[g][b], cudaEventDisableTiming);
    }
  }
  if (cudaGetLastError() != cudaSuccess) return LSPCA_ERR_CUDA;
  *out = s;
  return LSPCA_OK;
}

int lspca_srv_destroy(lspca_srv* s) {
  if (!s) return LSPCA_ERR_INVALID;
  cudaSetDevice(s->device);
  cudaStreamSynchronize(s->stream);
  cudaStreamSynchronize(s->pstream);
  for (int g = 0; g < kGroups; ++g) {
    for (int b = 0; b < 2; ++b) {
      if (s->gexec[g][b]) cudaGraphExecDestroy(s->gexec[g][b]);
      cudaFreeHost(s->h_units[g][b]);
      cudaFreeHost(s->h_count[g][b]);
      cudaEventDestroy(s->buf_ev[g][b]);
    }
    cudaFree(s->d_units[g]);
    cudaFree(s->d_count[g]);
  }
  for (auto& kv : s->reqs)
    if (kv.second.ev) s->ev_pool.push_back(kv.second.ev);
  std::sort(s->ev_pool.begin(), s->ev_pool.end());
  s->ev_pool.erase(std::unique(s->ev_pool.begin(), s->ev_pool.end()), s->ev_pool.end());
  for (auto e : s->ev_pool) cudaEventDestroy(e);
  cudaFree(s->arena);
  cudaFree(s->d_status);
  cudaStreamDestroy(s->stream);
  cudaStreamDestroy(s->pstream);
  delete s;
  return LSPCA_OK;
}

int lspca_srv_register_v(lspca_srv* s, const float* V, int64_t n, int32_t k, int32_t* v_id) {
  if (!s || !V || !v_id || n < 1 || k < 4 || k > 256 || (k % 4) != 0) return LSPCA_ERR_INVALID;
  if (((uintptr_t)V & 15u) != 0) return LSPCA_ERR_INVALID;
  SrvV e;
  e.V = V;
  e.n = n;
  e.k = k;
  s->vs.push_back(e);
  *v_id = (int32_t)(s->vs.size() - 1);
  return LSPCA_OK;
}

int lspca_srv_submit_project(lspca_srv* s, int32_t v_id, const void* X, int32_t xt, int64_t rows, int64_t ldx,
                             float* Y, int64_t* req) {
  if (!s || !X || !Y || !req || v_id < 0 || v_id >= (int32_t)s->vs.size() || rows < 1) return LSPCA_ERR_INVALID;
  const SrvV& v = s->vs[v_id];
  if (xt == LSPCA_F64 || xt < 0 || xt > LSPCA_E4M3 || ldx < v.n) return LSPCA_ERR_INVALID;
  if (((uintptr_t)X & 15u) || (ldx * (int64_t)dtype_size(xt)) % 16 != 0 || !tc_ok(xt, v.k)) return LSPCA_ERR_INVALID;
  Req r;
  r.id = s->next_id++;
  r.kind = KIND_PROJECT;
  r.X = X;
  r.xt = xt;
  r.rows = rows;
  r.ldx = ldx;
  r.n = v.n;
  r.k = v.k;
  r.v = v_id;
  r.Y = Y;
  s->reqs[r.id] = r;
  s->queue.push_back(r.id);
  *req = r.id;
  return LSPCA_OK;
}

int lspca_srv_submit_fit(lspca_srv* s, const void* X, int32_t xt, int64_t m, int64_t n, int64_t ldx, int32_t k,
                         lspca_omega om, float* V, double* sigma, int64_t* req) {
  if (!s || !X || !V || !sigma || !req || m < k || n < k || ldx < n || !tc_ok(xt, k)) return LSPCA_ERR_INVALID;
  if (((uintptr_t)X & 15u) || (ldx * (int64_t)dtype_size(xt)) % 16 != 0) return LSPCA_ERR_INVALID;
  if (om.kind != LSPCA_OMEGA_GAUSSIAN && om.kind != LSPCA_OMEGA_VERY_SPARSE) return LSPCA_ERR_INVALID;
  if (om.kind == LSPCA_OMEGA_VERY_SPARSE && om.p == 0) return LSPCA_ERR_INVALID;
  if (xt == LSPCA_E4M3 && om.kind != LSPCA_OMEGA_VERY_SPARSE) return LSPCA_ERR_INVALID;
  Req r;
  r.id = s->next_id++;
  r.kind = KIND_FIT;
  r.X = X;
  r.xt = xt;
  r.rows = m;
  r.n = n;
  r.ldx = ldx;
  r.k = k;
  r.om = om;
  r.Vout = V;
  r.sigma = sigma;
  r.ws_bytes = fit_layout(r, s->num_sms).total;
  if (r.ws_bytes > s->arena_size) return LSPCA_ERR_NOMEM;
  s->reqs[r.id] = r;
  s->queue.push_back(r.id);
  *req = r.id;
  return LSPCA_OK;
}

int lspca_srv_step(lspca_srv* s, int32_t* work_units) {
  if (!s) return LSPCA_ERR_INVALID;
  if (cudaSetDevice(s->device) != cudaSuccess) return LSPCA_ERR_CUDA;
  Launcher L{s->stream, &s->launches, s->num_sms};    // fits
  Launcher Lp{s->pstream, &s->launches, s->num_sms};  // projections
  retire(s);
  // 1. admission, FIFO: a slot, and for fits an arena block
  while (!s->queue.empty() && s->inflight < s->max_inflight) {
    Req& r = s->reqs[s->queue.front()];
    if (r.kind == KIND_FIT && !arena_alloc(s, r.ws_bytes, &r.ws_off)) break;
    r.state = REQ_RUNNING;
    s->inflight++;
    s->running.push_back(r.id);
    s->queue.pop_front();
  }
  int units = 0;
  // 2. projection tiles of all running projections, grouped by (X type, padded k)
  int cnt[kGroups] = {};
  std::vector<int64_t> finishing, pfinishing;
  for (int64_t id : s->running) {
    Req& r = s->reqs[id];
    if (r.kind != KIND_PROJECT || r.finishing) continue;
    SrvV& v = s->vs[r.v];
    const int xi = r.xt == LSPCA_F32 ? 0 : (r.xt == LSPCA_BF16 ? 1 : 2);
    if (!v.ready[xi]) {
      size_t off;
      const size_t bytes = tc_tile_v_bytes(v.n, v.k) + 256;
      if (!arena_alloc(s, bytes, &off)) continue;  // wait for memory
      v.tiles_off[xi] = off;
      tc_tile_v(Lp, r.xt, v.V, v.n, v.k, s->arena + off + 256, (float*)(s->arena + off), s->d_status);
      v.ready[xi] = true;
    }
    const int g = group_of(r.xt, r.k);
    const int b = s->flip[g];
    if (cnt[g] == 0) cudaEventSynchronize(s->buf_ev[g][b]);  // host table free again
    TcProjUnit* tab = s->h_units[g][b];
    while (r.next < r.rows && cnt[g] < kMaxTiles) {
      TcProjUnit& u = tab[cnt[g]++];
      u.X = r.X;
      u.ldx = r.ldx;
      u.m = r.rows;
      u.row0 = r.next;
      u.n = v.n;
      u.k = v.k;
      u.pad = 0;
      u.vt = (const uint8_t*)(s->arena + v.tiles_off[xi] + 256);
      u.vscale = (const float*)(s->arena + v.tiles_off[xi]) + 1;
      u.Y = r.Y;
      r.next += 128;
    }
    if (r.next >= r.rows) {
      r.finishing = true;
      pfinishing.push_back(id);
    }
  }
  for (int g = 0; g < kGroups; ++g) {
    if (!cnt[g]) continue;
    const int b = s->flip[g];
    *s->h_count[g][b] = cnt[g];
    units += cnt[g];
    const int xt = g / 4 == 0 ? LSPCA_F32 : (g / 4 == 1 ? LSPCA_BF16 : LSPCA_E4M3);
    const int k = (g % 4 + 1) * 64;
    if (!s->warmed[g]) {
      // first batch of the group: direct launch (sets kernel attributes), then capture
      cudaMemcpyAsync(s->d_units[g], s->h_units[g][b], sizeof(TcProjUnit) * kMaxTiles, cudaMemcpyHostToDevice,
                      s->pstream);
      cudaMemcpyAsync(s->d_count[g], s->h_count[g][b], sizeof(int), cudaMemcpyHostToDevice, s->pstream);
      tc_project_batch(Lp, xt, k, s->d_units[g], s->d_count[g], kMaxTiles, s->d_status);
      for (int bb = 0; bb < 2; ++bb) {
        cudaGraph_t graph = nullptr;
        int64_t dummy = 0;
        Launcher Lc{s->pstream, &dummy, s->num_sms};
        if (cudaStreamBeginCapture(s->pstream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) break;
        cudaMemcpyAsync(s->d_units[g], s->h_units[g][bb], sizeof(TcProjUnit) * kMaxTiles, cudaMemcpyHostToDevice,
                        s->pstream);
        cudaMemcpyAsync(s->d_count[g], s->h_count[g][bb], sizeof(int), cudaMemcpyHostToDevice, s->pstream);
        tc_project_batch(Lc, xt, k, s->d_units[g], s->d_count[g], kMaxTiles, s->d_status);
        if (cudaStreamEndCapture(s->pstream, &graph) != cudaSuccess || !graph) break;
        if (cudaGraphInstantiate(&s->gexec[g][bb], graph, 0) != cudaSuccess) s->gexec[g][bb] = nullptr;
        cudaGraphDestroy(graph);
      }
      cudaGetLastError();
      s->warmed[g] = true;
    } else if (s->gexec[g][b]) {
      cudaGraphLaunch(s->gexec[g][b], s->pstream);
      s->launches += 1;
    } else {
      cudaMemcpyAsync(s->d_units[g], s->h_units[g][b], sizeof(TcProjUnit) * kMaxTiles, cudaMemcpyHostToDevice,
                      s->pstream);
      cudaMemcpyAsync(s->d_count[g], s->h_count[g][b], sizeof(int), cudaMemcpyHostToDevice, s->pstream);
      tc_project_batch(Lp, xt, k, s->d_units[g], s->d_count[g], kMaxTiles, s->d_status);
    }
    cudaEventRecord(s->buf_ev[g][b], s->pstream);
    s->flip[g] ^= 1;
  }
  // 3. one Algorithm-4 slice of every running fit
  for (int64_t id : s->running) {
    Req& r = s->reqs[id];
    if (r.kind != KIND_FIT || r.finishing) continue;
    if (!r.prepared) fit_prepare(s, r, L);
    if (!fit_slice(s, r, L)) return LSPCA_ERR_CUDA;
    units += 1;
    if (r.finishing) finishing.push_back(id);
  }
  // 4. completion events of the requests this batch finishes (one event each,
  //    recorded after the batch's last launch on the request's stream)
  for (int64_t id : pfinishing) {
    Req& r = s->reqs[id];
    r.ev = take_event(s);
    cudaEventRecord(r.ev, s->pstream);
  }
  for (int64_t id : finishing) {
    Req& r = s->reqs[id];
    r.ev = take_event(s);
    cudaEventRecord(r.ev, s->stream);
  }
  if (work_units) *work_units = units;
  return cudaGetLastError() == cudaSuccess ? LSPCA_OK : LSPCA_ERR_CUDA;
}

int lspca_srv_poll(lspca_srv* s, int64_t req, int32_t* done) {
  if (!s || !done) return LSPCA_ERR_INVALID;
  if (cudaSetDevice(s->device) != cudaSuccess) return LSPCA_ERR_CUDA;
  retire(s);
  auto it = s->reqs.find(req);
  if (it == s->reqs.end()) return LSPCA_ERR_INVALID;
  Req& r = it->second;
  if (r.state == REQ_DONE) {
    *done = 1;
    return LSPCA_OK;
  }
  *done = (r.finishing && r.ev && cudaEventQuery(r.ev) == cudaSuccess) ? 1 : 0;
  cudaGetLastError();
  return LSPCA_OK;
}

int lspca_srv_wait(lspca_srv* s, int64_t req, int32_t timeout_ms) {
  if (!s) return LSPCA_ERR_INVALID;
  const auto t0 = std::chrono::steady_clock::now();
  while (true) {
    int32_t d = 0;
    int st = lspca_srv_poll(s, req, &d);
    if (st) return st;
    if (d) return LSPCA_OK;
    const Req& r = s->reqs[req];
    if (!r.finishing) {
      // not yet scheduled to completion: drive the server
      int32_t u = 0;
      if ((st = lspca_srv_step(s, &u))) return st;
    } else {
      std::this_thread::sleep_for(std::chrono::microseconds(20));
    }
    const double ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    if (ms > timeout_ms) return LSPCA_ERR_TIMEOUT;
  }
}

int lspca_srv_release(lspca_srv* s, int64_t req) {
  if (!s) return LSPCA_ERR_INVALID;
  retire(s);
  auto it = s->reqs.find(req);
  if (it == s->reqs.end()) return LSPCA_ERR_INVALID;
  if (it->second.state != REQ_DONE) return LSPCA_ERR_BUSY;
  s->reqs.erase(it);
  return LSPCA_OK;
}

int64_t lspca_srv_launch_count(lspca_srv* s) { return s ? s->launches : 0; }

}  // extern "C"
