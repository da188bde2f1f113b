// lspca_chain_noalloc: pass F (F = U^T X) on tensor cores without allocating.
//
// Some callers cannot allocate device memory at all: code that runs inside a
// host framework which owns every byte of the GPU through its own pool and
// forbids allocations behind its back, or latency-critical loops that cannot
// afford the implicit device synchronisation of cudaMalloc/cudaFree.  For them
// this entry point takes its scratch -- the FP32 partial sums of the m-chunks,
// the two max|.| scalars that set the split-FP16 scales, and a status word --
// from a file-scope device array of fixed size instead of a library workspace.
//
// Properties of the array:
// * every GPU that loads the library holds the array (kNoallocScratchBytes)
//   until the process exits;
// * host code cannot use the array's name as a device address (in host code it
//   is a host-side stand-in), so the device address is fetched with
//   cudaGetSymbolAddress once per device, with that device current, by the
//   first call on that device -- that first call should therefore come before
//   any stream capture;
// * every call on a device shares the array and it keeps the last call's
//   contents: the scalars that must start at zero are cleared with
//   cudaMemsetAsync on the caller's stream; calls whose executions overlap on
//   the GPU (different streams, no ordering) race on the array.
#include <mutex>

#include "common.cuh"
#include "kernels.h"
#include "tc.h"

namespace lspca {

constexpr size_t kNoallocScratchBytes = (size_t)16 << 20;  // 16 MiB
constexpr size_t kNoallocHeader = 256;                      // absmax[2] + status

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocScratchBytes];

namespace {
constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_addr[kMaxDevices] = {};
int g_sms[kMaxDevices] = {};

// Device address of the scratch array on the current device (set up once).
int scratch_address(int dev, void** out, int* sms) {
  if (dev < 0 || dev >= kMaxDevices) return LSPCA_ERR_INVALID;
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_addr[dev]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || p == nullptr) {
      cudaGetLastError();
      return LSPCA_ERR_CUDA;
    }
    int n = 0;
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return LSPCA_ERR_CUDA;
    g_addr[dev] = p;
    g_sms[dev] = n;
  }
  *out = g_addr[dev];
  *sms = g_sms[dev];
  return LSPCA_OK;
}
}  // namespace

}  // namespace lspca

using namespace lspca;

extern "C" int lspca_chain_noalloc(const void* X, int32_t xt, int64_t m, int64_t n, int64_t ldx, const float* U,
                                   int32_t k, double* F, int32_t* status, void* stream) {
  if (!X || !U || !F) return LSPCA_ERR_INVALID;
  if (xt != LSPCA_F32 && xt != LSPCA_BF16) return LSPCA_ERR_INVALID;
  if (m < 1 || n < 1 || ldx < n || k < 4 || k > 256 || (k % 4) != 0) return LSPCA_ERR_INVALID;
  if (((uintptr_t)X & 15u) || ((uintptr_t)U & 15u) || (ldx * (int64_t)dtype_size(xt)) % 16 != 0)
    return LSPCA_ERR_INVALID;
  if (!tc_available()) return LSPCA_ERR_INVALID;
  // one m-chunk needs k x n FP32 partials in the array
  const size_t part_cap = kNoallocScratchBytes - kNoallocHeader;
  const size_t per_chunk = (size_t)k * (size_t)n * 4;
  if (per_chunk > part_cap) return LSPCA_ERR_NOMEM;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return LSPCA_ERR_CUDA;
  void* base = nullptr;
  int sms = 0;
  int st = scratch_address(dev, &base, &sms);
  if (st) return st;
  cudaStream_t s = (cudaStream_t)stream;
  int64_t launches = 0;  // per call: nothing reads it, and calls may come from several threads
  Launcher L{s, &launches, sms};

  float* absmax = reinterpret_cast<float*>(base);
  int* dstatus = status ? reinterpret_cast<int*>(status) : reinterpret_cast<int*>((char*)base + 64);
  // chunking of the regular pass, capped by the array's capacity
  TcChainWs w;
  plan_tc_chain_inline(nullptr, w, xt, m, n, k, false, sms);
  int64_t chunks = w.chunks;
  const int64_t cap_chunks = (int64_t)(part_cap / per_chunk);
  if (chunks > cap_chunks) {
    int64_t rows = (m + cap_chunks - 1) / cap_chunks;
    rows = (rows + 31) / 32 * 32;
    w.rows_per_chunk = rows;
    chunks = (m + rows - 1) / rows;
  }
  w.chunks = (int)chunks;
  w.Fpart = reinterpret_cast<double*>((char*)base + kNoallocHeader);
  w.Gpart = nullptr;
  w.gchunks = 0;

  if (cudaMemsetAsync(base, 0, 64, s) != cudaSuccess) return LSPCA_ERR_CUDA;
  if (cudaMemsetAsync(dstatus, 0, sizeof(int), s) != cudaSuccess) return LSPCA_ERR_CUDA;
  // max|X| (the FP16 scale for FP32 X) and the non-finite check of X, as lspca_chain does
  launch_scan_x(L, X, xt, m, n, ldx, absmax, dstatus);
  if (xt == LSPCA_F32) launch_scan_x(L, U, LSPCA_F32, m, k, k, absmax + 1, dstatus);
  tc_chain_inline_main(L, X, xt, m, n, ldx, U, k, w, absmax, dstatus, false);
  tc_chain_reduce(L, n, k, w, F, nullptr);
  return cudaGetLastError() == cudaSuccess ? LSPCA_OK : LSPCA_ERR_CUDA;
}
