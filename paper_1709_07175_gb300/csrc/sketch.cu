// K1, pass S for the very sparse Omega (Sec. I-A): U = X Omega (Eq. 1, c = 1).
//
// U[r, c] = sum over the nonzeros (j, s) of column c of Omega of s * X[r, j].
// Omega has about n/p nonzeros per column, so the sketch is a gather-add: it
// is bound by streaming X from HBM, not by arithmetic.
//
// One persistent CTA per SM (512 threads) walks row tiles of 32 rows; each tile
// is streamed in column chunks of W elements with 16-byte loads held in
// registers one step ahead.  A chunk is stored transposed, Xt[j][r] with a
// pitch of 33, so that the gather -- lane = row, all lanes reading the same
// feature j -- is free of bank conflicts; the lane mapping of the stores
// (EPV rows x 32/EPV vectors per warp instruction, EPV = elements per vector)
// makes the transposing stores conflict-free as well.  Each warp owns the Omega
// columns c = warp + 16 t and walks their sorted index lists, one entry per
// column per round so that the lists' loads overlap.  A finished tile is staged
// through shared memory and written with coalesced row stores.
//
// Summation of each U entry runs over j in increasing order in the
// accumulation type (FP64 for FP64 X, else FP32): deterministic.
#include "common.cuh"
#include "kernels.h"
#include "tc_ptx.cuh"
#include "tma.h"

namespace lspca {

template <int DT>
struct SketchCfg {
  using T = typename XType<DT>::T;
  using Acc = typename XType<DT>::Acc;
  static constexpr int EPV = 16 / (int)sizeof(T);               // elements per 16-byte vector
  static constexpr int W = sizeof(Acc) == 8 ? 128 : 512;         // chunk width in elements
  static constexpr int ROWS = 32;
  static constexpr int THREADS = 512;
  static constexpr int VPT = ROWS * W / EPV / THREADS;           // vectors per thread per chunk
  static constexpr int RG = 32 / EPV;                            // row groups per chunk
  static constexpr int PITCH = ROWS + 1;
  static constexpr int MAX_CPW = 16;                             // k <= 256 -> 16 columns per warp
  static constexpr int ENT_CACHE = 12288;                        // Omega entries cached in SMEM (int16)
  static constexpr int OFF_CACHE = 4096;                         // (column, chunk) offsets in SMEM
  static size_t smem_bytes(int k) {
    return (size_t)(2 * W * PITCH + ROWS * (k + 1)) * sizeof(Acc) + (size_t)ENT_CACHE * 2 + (size_t)OFF_CACHE * 4;
  }
};

__device__ __forceinline__ float4 ldg_nc_na(const void* p) {
  float4 v;
  asm volatile("ld.global.nc.L1::no_allocate.v4.f32 {%0, %1, %2, %3}, [%4];"
               : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
               : "l"(p));
  return v;
}

// Entry encoding in the CSC lists: e = s * (j + 1).  The kernel needs, for
// every column c and chunk q, the first list position with j >= q W; it builds
// that table in shared memory (one thread per column) when it fits, so the
// gather of a chunk walks fixed ranges [off(c, q), off(c, q + 1)).
template <int DT>
__global__ void __launch_bounds__(512, 1)
    sketch_sparse_kernel(const void* __restrict__ Xv, int64_t m, int64_t n, int64_t ldx, int k,
                         const int32_t* __restrict__ col_ptr, const int32_t* __restrict__ entries_g,
                         int32_t* __restrict__ off_g, void* __restrict__ Uv, int64_t ldu, float* absmax, int* status) {
  using C = SketchCfg<DT>;
  using T = typename C::T;
  using Acc = typename C::Acc;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Acc* buf0 = reinterpret_cast<Acc*>(smem_raw);
  Acc* buf1 = buf0 + C::W * C::PITCH;
  Acc* us = buf1 + C::W * C::PITCH;
  int16_t* ent_s = reinterpret_cast<int16_t*>(us + C::ROWS * (k + 1));
  int32_t* off_s = reinterpret_cast<int32_t*>(ent_s + C::ENT_CACHE);

  const T* X = reinterpret_cast<const T*>(Xv);
  Acc* U = reinterpret_cast<Acc*>(Uv);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int rr = lane % C::EPV, cc = lane / C::EPV;
  const int nchunks = (int)((n + C::W - 1) / C::W);
  const int noff = k * (nchunks + 1);

  // Omega lists: int16 copies in SMEM when they fit (n < 32767), else global.
  const int nnz = col_ptr[k];
  const bool ent_in_smem = nnz <= C::ENT_CACHE && n < 32767;
  if (ent_in_smem)
    for (int e = tid; e < nnz; e += C::THREADS) ent_s[e] = (int16_t)entries_g[e];
  // chunk offsets: SMEM table when small, else a global table (built once per call)
  int32_t* off = (noff <= C::OFF_CACHE) ? off_s : off_g;
  for (int c = tid; c < k; c += C::THREADS) {
    int pos = col_ptr[c];
    const int end = col_ptr[c + 1];
    for (int q = 0; q <= nchunks; ++q) {
      const int64_t lim = (int64_t)q * C::W;
      while (pos < end) {
        const int e = entries_g[pos];
        if ((int64_t)((e > 0 ? e : -e) - 1) >= lim) break;
        ++pos;
      }
      off[c * (nchunks + 1) + q] = pos;
    }
    off[c * (nchunks + 1) + nchunks] = end;
  }

  const int64_t ntiles = (m + C::ROWS - 1) / C::ROWS;
  const int64_t my_tiles = ((int64_t)blockIdx.x < ntiles) ? (ntiles - blockIdx.x + gridDim.x - 1) / gridDim.x : 0;
  const int64_t steps = my_tiles * nchunks;
  __syncthreads();
  if (steps == 0) return;

  float4 regs[C::VPT];
  float amax = 0.f, amax_u = 0.f;
  bool bad = false;
  Acc acc[C::MAX_CPW];

  auto load = [&](int64_t tile, int chunk) {
    const int64_t r0 = tile * C::ROWS;
    const int64_t j0 = (int64_t)chunk * C::W;
#pragma unroll
    for (int q = 0; q < C::VPT; ++q) {
      const int s = q * 16 + warp;
      const int row = (s % C::RG) * C::EPV + rr;
      const int vc = (s / C::RG) * (32 / C::EPV) + cc;
      const int64_t gr = r0 + row, gj = j0 + (int64_t)vc * C::EPV;
      if (gr < m && gj < n)
        regs[q] = ldg_nc_na(X + gr * ldx + gj);
      else
        regs[q] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
  };

  auto store = [&](int chunk, Acc* buf) {
    const int64_t j0 = (int64_t)chunk * C::W;
#pragma unroll
    for (int q = 0; q < C::VPT; ++q) {
      const int s = q * 16 + warp;
      const int row = (s % C::RG) * C::EPV + rr;
      const int vc = (s / C::RG) * (32 / C::EPV) + cc;
      const T* e = reinterpret_cast<const T*>(&regs[q]);
#pragma unroll
      for (int u = 0; u < C::EPV; ++u) {
        const int jl = vc * C::EPV + u;
        Acc v = XType<DT>::to_acc(e[u]);
        if (j0 + jl >= n) v = Acc(0);
        if (!finite_acc(v)) bad = true;
        amax = fmaxf(amax, (float)abs_acc(v));
        buf[jl * C::PITCH + row] = v;
      }
    }
  };

  const int cpw = (k + 15) / 16;
  int64_t tile = blockIdx.x;
  int chunk = 0;
  load(tile, chunk);
  store(chunk, buf0);
  __syncthreads();
  for (int64_t st = 0; st < steps; ++st) {
    Acc* cur = (st & 1) ? buf1 : buf0;
    Acc* nxt = (st & 1) ? buf0 : buf1;
    const int j0 = chunk * C::W;
    if (chunk == 0) {
#pragma unroll
      for (int t = 0; t < C::MAX_CPW; ++t) acc[t] = Acc(0);
    }
    int64_t ntile = tile;
    int nchunk = chunk + 1;
    if (nchunk == nchunks) {
      nchunk = 0;
      ntile += gridDim.x;
    }
    if (st + 1 < steps) load(ntile, nchunk);
    // gather: for each owned column, the fixed range of its entries in this chunk
#pragma unroll
    for (int t = 0; t < C::MAX_CPW; ++t) {
      const int c = warp + 16 * t;
      if (t < cpw && c < k) {
        const int b = off[c * (nchunks + 1) + chunk];
        const int e = off[c * (nchunks + 1) + chunk + 1];
        Acc a = acc[t];
        if (ent_in_smem) {
#pragma unroll 4
          for (int i = b; i < e; ++i) {
            const int en = ent_s[i];
            const Acc v = cur[((en > 0 ? en : -en) - 1 - j0) * C::PITCH + lane];
            a += (en > 0) ? v : -v;
          }
        } else {
#pragma unroll 4
          for (int i = b; i < e; ++i) {
            const int en = __ldg(entries_g + i);
            const Acc v = cur[((en > 0 ? en : -en) - 1 - j0) * C::PITCH + lane];
            a += (en > 0) ? v : -v;
          }
        }
        acc[t] = a;
      }
    }
    const bool last = (chunk == nchunks - 1);
    if (last) {
#pragma unroll
      for (int t = 0; t < C::MAX_CPW; ++t) {
        const int c = warp + 16 * t;
        if (t < cpw && c < k) us[lane * (k + 1) + c] = acc[t];
      }
    }
    if (st + 1 < steps) store(nchunk, nxt);
    __syncthreads();
    if (last) {
      const int64_t r0 = tile * C::ROWS;
      for (int e = tid; e < C::ROWS * k; e += C::THREADS) {
        const int r = e / k, c = e % k;
        if (r0 + r < m) {
          const Acc v = us[r * (k + 1) + c];
          amax_u = fmaxf(amax_u, (float)abs_acc(v));
          U[(r0 + r) * ldu + c] = v;
        }
      }
      __syncthreads();
    }
    tile = ntile;
    chunk = nchunk;
  }
  amax = warp_max(amax);
  amax_u = warp_max(amax_u);
  const unsigned anybad = __ballot_sync(0xffffffffu, bad);
  if (lane == 0) {
    atomic_max_nonneg(absmax, amax);
    atomic_max_nonneg(absmax + 1, amax_u);
    if (anybad) atomicOr(status, ST_NONFINITE);
  }
}

// ---------------------------------------------------------------------------
// Wide variant for 4-byte accumulation (FP32/BF16/E4M3 X) and k <= 128.
//
// Tiles of 128 rows; each lane owns 4 consecutive rows, so one 16-byte shared
// load of Xt[j][4 lane .. 4 lane + 3] serves 4 rows of one gather.  Chunks of
// W4 = 128 columns; Xt pitch 132 floats (16-byte aligned rows).  The global
// loads of a warp instruction cover 16 rows x 2 vectors, which makes the
// transposing 4-byte stores bank-conflict-free for FP32 (2-way for 2- and
// 1-byte types).  The Omega entries of every (column, chunk) are re-encoded in
// shared memory as the byte offset of row j of the chunk, with the sign in bit
// 31, so a gather is: load code, mask, 16-byte load, sign, four FMAs.
// NaN/Inf detection and max|X| use one integer max over |bits| per element.
constexpr int W4 = 128;
constexpr int P4 = 132;
constexpr int R4 = 128;
constexpr int ENT4 = 10240;
constexpr int OFF4 = 4608;

static size_t smem4_bytes() { return (size_t)2 * W4 * P4 * 4 + (size_t)ENT4 * 4 + (size_t)OFF4 * 4; }

template <int DT>
__global__ void __launch_bounds__(512, 1)
    sketch_sparse4_kernel(const void* __restrict__ Xv, int64_t m, int64_t n, int64_t ldx, int k,
                          const int32_t* __restrict__ col_ptr, const int32_t* __restrict__ entries_g,
                          int32_t* __restrict__ off_g, int32_t* __restrict__ code_g, float* __restrict__ U,
                          int64_t ldu, float* absmax, int* status) {
  using T = typename XType<DT>::T;
  constexpr int EPV = 16 / (int)sizeof(T);
  constexpr int VPT = R4 * W4 / EPV / 512;  // 16-byte vectors per thread per chunk
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float* buf0 = reinterpret_cast<float*>(smem_raw);
  float* buf1 = buf0 + W4 * P4;
  int32_t* code_s = reinterpret_cast<int32_t*>(buf1 + W4 * P4);
  int32_t* off_s = code_s + ENT4;

  const T* X = reinterpret_cast<const T*>(Xv);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int nchunks = (int)((n + W4 - 1) / W4);
  const int noff = k * (nchunks + 1);
  const int nnz = col_ptr[k];
  const bool code_in_smem = nnz <= ENT4;
  int32_t* codes = code_in_smem ? code_s : code_g;
  int32_t* off = (noff <= OFF4) ? off_s : off_g;
  // re-encode: code = sign bit | byte offset of row (j mod W4) inside a chunk buffer
  for (int e = tid; e < nnz; e += 512) {
    const int en = entries_g[e];
    const int j = (en > 0 ? en : -en) - 1;
    codes[e] = (en < 0 ? (int)0x80000000 : 0) | ((j % W4) * P4 * 4);
  }
  for (int c = tid; c < k; c += 512) {
    int pos = col_ptr[c];
    const int end = col_ptr[c + 1];
    for (int q = 0; q < nchunks; ++q) {
      off[c * (nchunks + 1) + q] = pos;
      const int64_t lim = (int64_t)(q + 1) * W4;
      while (pos < end) {
        const int en = entries_g[pos];
        if ((int64_t)((en > 0 ? en : -en) - 1) >= lim) break;
        ++pos;
      }
    }
    off[c * (nchunks + 1) + nchunks] = end;
  }
  const int64_t ntiles = (m + R4 - 1) / R4;
  const int64_t my_tiles = ((int64_t)blockIdx.x < ntiles) ? (ntiles - blockIdx.x + gridDim.x - 1) / gridDim.x : 0;
  const int64_t steps = my_tiles * nchunks;
  __syncthreads();
  if (steps == 0) return;

  // per-thread load slots: warp-instruction slot s = q * 16 + warp covers rows
  // (s % 8) * 16 + (lane % 16) and vector column (s / 8) * 2 + lane / 16
  const int lr = lane & 15, lh = lane >> 4;
  uint4 regs[VPT];
  uint32_t mxb = 0u;
  float acc[8][4];
  const int cpw = (k + 15) / 16;

  auto load = [&](int64_t tile, int chunk) {
    const int64_t r0 = tile * R4, j0 = (int64_t)chunk * W4;
#pragma unroll
    for (int q = 0; q < VPT; ++q) {
      const int s = q * 16 + warp;
      const int row = (s % 8) * 16 + lr;
      const int vc = (s / 8) * 2 + lh;
      const int64_t gr = r0 + row, gj = j0 + (int64_t)vc * EPV;
      if (gr < m && gj < n)
        asm volatile("ld.global.nc.L1::no_allocate.v4.u32 {%0, %1, %2, %3}, [%4];"
                     : "=r"(regs[q].x), "=r"(regs[q].y), "=r"(regs[q].z), "=r"(regs[q].w)
                     : "l"(X + gr * ldx + gj));
      else
        regs[q] = make_uint4(0u, 0u, 0u, 0u);
    }
  };
  auto store = [&](int chunk, float* buf) {
    const int64_t j0 = (int64_t)chunk * W4;
    const bool tail = j0 + W4 > n;
#pragma unroll
    for (int q = 0; q < VPT; ++q) {
      const int s = q * 16 + warp;
      const int row = (s % 8) * 16 + lr;
      const int vc = (s / 8) * 2 + lh;
      const T* e = reinterpret_cast<const T*>(&regs[q]);
#pragma unroll
      for (int u = 0; u < EPV; ++u) {
        const int jl = vc * EPV + u;
        float v = XType<DT>::to_acc(e[u]);
        if (tail && j0 + jl >= n) v = 0.f;
        mxb = max(mxb, __float_as_uint(v) & 0x7fffffffu);
        buf[jl * P4 + row] = v;
      }
    }
  };

  int64_t tile = blockIdx.x;
  int chunk = 0;
  load(tile, chunk);
  store(chunk, buf0);
  __syncthreads();
  for (int64_t st = 0; st < steps; ++st) {
    float* cur = (st & 1) ? buf1 : buf0;
    float* nxt = (st & 1) ? buf0 : buf1;
    if (chunk == 0) {
#pragma unroll
      for (int t = 0; t < 8; ++t)
#pragma unroll
        for (int r = 0; r < 4; ++r) acc[t][r] = 0.f;
    }
    int64_t ntile = tile;
    int nchunk = chunk + 1;
    if (nchunk == nchunks) {
      nchunk = 0;
      ntile += gridDim.x;
    }
    if (st + 1 < steps) load(ntile, nchunk);
    const char* cur_lane = reinterpret_cast<const char*>(cur) + lane * 16;
#pragma unroll
    for (int t = 0; t < 8; ++t) {
      const int c = warp + 16 * t;
      if (t < cpw && c < k) {
        const int b = off[c * (nchunks + 1) + chunk];
        const int e = off[c * (nchunks + 1) + chunk + 1];
        float a0 = acc[t][0], a1 = acc[t][1], a2 = acc[t][2], a3 = acc[t][3];
#pragma unroll 4
        for (int i = b; i < e; ++i) {
          const int code = codes[i];
          const float4 v = *reinterpret_cast<const float4*>(cur_lane + (code & 0x7fffffff));
          const float sg = __int_as_float((code & (int)0x80000000) | 0x3f800000);
          a0 = fmaf(sg, v.x, a0);
          a1 = fmaf(sg, v.y, a1);
          a2 = fmaf(sg, v.z, a2);
          a3 = fmaf(sg, v.w, a3);
        }
        acc[t][0] = a0;
        acc[t][1] = a1;
        acc[t][2] = a2;
        acc[t][3] = a3;
      }
    }
    const bool last = (chunk == nchunks - 1);
    if (st + 1 < steps) store(nchunk, nxt);
    __syncthreads();
    if (last) {
      // stage the tile's U through the buffer just consumed (free until the next
      // step's store) and write rows coalesced
      float* us = cur;
      const int ldp = k + 1;
#pragma unroll
      for (int t = 0; t < 8; ++t) {
        const int c = warp + 16 * t;
        if (t < cpw && c < k) {
#pragma unroll
          for (int r = 0; r < 4; ++r) us[(4 * lane + r) * ldp + c] = acc[t][r];
        }
      }
      __syncthreads();
      const int64_t r0 = tile * R4;
      float umx = 0.f;
      for (int e = tid; e < R4 * k; e += 512) {
        const int r = e / k, c = e - r * k;
        if (r0 + r < m) {
          const float v = us[r * ldp + c];
          umx = fmaxf(umx, fabsf(v));
          U[(r0 + r) * ldu + c] = v;
        }
      }
      umx = warp_max(umx);
      if (lane == 0) atomic_max_nonneg(absmax + 1, umx);
      __syncthreads();
    }
    tile = ntile;
    chunk = nchunk;
  }
  // one integer max over |bits| covers both max|X| and NaN/Inf (bits >= 0x7f800000)
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) mxb = max(mxb, __shfl_xor_sync(0xffffffffu, mxb, o));
  if (lane == 0) {
    if (mxb >= 0x7f800000u) atomicOr(status, ST_NONFINITE);
    else atomic_max_nonneg(absmax, __uint_as_float(mxb));
  }
}

template <int DT>
static bool sketch_sparse4_dispatch(Launcher& L, const void* X, int64_t m, int64_t n, int64_t ldx, int k,
                                    const int32_t* col_ptr, const int32_t* entries, int32_t* off, int32_t* codes,
                                    float* U, int64_t ldu, float* absmax, int* status) {
  if (k > 128) return false;
  const size_t smem = smem4_bytes();
  cudaFuncSetAttribute(sketch_sparse4_kernel<DT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  const int64_t ntiles = (m + R4 - 1) / R4;
  const int grid = (int)(ntiles < L.num_sms ? ntiles : L.num_sms);
  sketch_sparse4_kernel<DT><<<grid, 512, smem, L.stream>>>(X, m, n, ldx, k, col_ptr, entries, off, codes, U, ldu,
                                                            absmax, status);
  L.count(1);
  return true;
}

template <int DT>
static void sketch_sparse_dispatch(Launcher& L, const void* X, int64_t m, int64_t n, int64_t ldx, int k,
                                   const int32_t* col_ptr, const int32_t* entries, int32_t* off, void* U, int64_t ldu,
                                   float* absmax, int* status) {
  using C = SketchCfg<DT>;
  const size_t smem = C::smem_bytes(k);
  cudaFuncSetAttribute(sketch_sparse_kernel<DT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  const int64_t ntiles = (m + C::ROWS - 1) / C::ROWS;
  const int grid = (int)(ntiles < L.num_sms ? ntiles : L.num_sms);
  sketch_sparse_kernel<DT><<<grid, C::THREADS, smem, L.stream>>>(X, m, n, ldx, k, col_ptr, entries, off, U, ldu,
                                                                  absmax, status);
  L.count(1);
}


// ---------------------------------------------------------------------------
// Streaming variant for FP32 / BF16 X and k <= 128 with an asynchronous copy
// ring (the form the dispatcher prefers).
//
// Row tiles of R5 = 128 rows are streamed in steps of W5 = 64 columns.  One
// thread issues each step as tiled TMA copies (boxes of 128 rows x 128 bytes
// with the 128-byte swizzle; rows past m and columns past n arrive as zeros)
// into a ring of S stages, S steps ahead, so the loads stay in flight while the
// CTA gathers.  With the swizzle, 8 consecutive rows at the same 16-byte
// column chunk fall on 8 different bank groups, so a warp reading 32 rows x 16
// bytes is conflict-free.  Each step the whole CTA transposes its stage into
// Xt[j][r] (FP32, pitch R5; consecutive lanes = consecutive rows, so the
// 4-byte stores are conflict-free) and then gathers from Xt exactly as the
// kernel above: lane = 4 consecutive rows, one 16-byte load per Omega entry.
// Xt is double-buffered, so one barrier per step orders the transpose of step
// s + 1 after every warp's gather of step s - 1, and the refill of a ring
// stage after every warp's transpose of it.  Warp w owns the Omega columns
// [w cpw, (w + 1) cpw), cpw = ceil(k / 16): a finished tile's row of U is cpw
// consecutive floats per thread, written as 16-byte stores.
// Entry codes are 16 bits: sign in bit 15, byte offset of row (j mod W5) of
// Xt in bits 0..14 (in shared memory when Omega has at most ENT5 nonzeros,
// else in a global scratch), stored chunk-major: the entries of (step chunk q,
// column c) follow those of (q, c - 1), ascending in j, so the begin offsets
// of a warp's cpw columns in a chunk are cpw + 1 consecutive words that lanes
// 0..cpw load at once and the gather loop receives by shuffles.
// A wait on a stage gives up after 2 s: the CTA records ST_TIMEOUT, waits
// (bounded) for its copies in flight and returns.
constexpr int R5 = 128;
constexpr int W5 = 64;
constexpr int ENT5 = 12288;
constexpr int PTR5 = 8704;  // max nch * k + 1 (chunk-major begin offsets)

template <int DT>
struct Sk5 {
  using T = typename XType<DT>::T;
  static constexpr int ELEM = (int)sizeof(T);
  static constexpr int BOXW = 128 / ELEM;              // columns per 128-byte swizzled box row
  static constexpr int NBOX = W5 / BOXW;               // boxes per step (2 for FP32, 1 for BF16)
  static constexpr int BOX_BYTES = R5 * 128;
  static constexpr int STAGE = NBOX * BOX_BYTES;
  static constexpr int S = ELEM == 4 ? 3 : 5;          // ring stages
  static constexpr int CHUNKS = W5 * ELEM / 16;        // 16-byte chunks per staged row
  static constexpr int EPC = 16 / ELEM;                // elements per chunk
  static constexpr size_t XT_OFF = (size_t)S * STAGE;
  static constexpr size_t CODE_OFF = XT_OFF + (size_t)2 * W5 * R5 * 4;
  static constexpr size_t PTR_OFF = CODE_OFF + (size_t)ENT5 * 2;
  static constexpr size_t RED_OFF = PTR_OFF + (size_t)PTR5 * 4;
  static constexpr size_t BAR_OFF = RED_OFF + 32 * 4;
  static constexpr size_t SMEM = 1024 + BAR_OFF + 8 * S;  // + alignment of the ring to 1024 bytes
};

template <int DT>
__global__ void __launch_bounds__(512, 1)
    sketch_sparse5_kernel(const __grid_constant__ CUtensorMap tmx, int64_t m, int64_t n, int k,
                          const int32_t* __restrict__ col_ptr, const int32_t* __restrict__ entries_g,
                          uint16_t* __restrict__ codes_g, float* __restrict__ U, int64_t ldu, int vec_u,
                          float* absmax, int* status) {
  using C = Sk5<DT>;
  using T = typename C::T;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  unsigned char* sm = reinterpret_cast<unsigned char*>(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  unsigned char* ring = sm;
  float* xt = reinterpret_cast<float*>(sm + C::XT_OFF);
  uint32_t* ptr = reinterpret_cast<uint32_t*>(sm + C::PTR_OFF);
  uint32_t* red = reinterpret_cast<uint32_t*>(sm + C::RED_OFF);
  uint64_t* full = reinterpret_cast<uint64_t*>(sm + C::BAR_OFF);

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int nch = (int)((n + W5 - 1) / W5);
  const int nnz = col_ptr[k];
  const int nslot = nch * k;  // (chunk, column) slots, chunk-major
  uint16_t* codes = nnz <= ENT5 ? reinterpret_cast<uint16_t*>(sm + C::CODE_OFF) : codes_g;
  // 1. entries per (chunk, column): thread c walks column c (its slots only)
  for (int i = tid; i <= nslot; i += 512) ptr[i] = 0u;
  __syncthreads();
  for (int c = tid; c < k; c += 512)
    for (int e = col_ptr[c]; e < col_ptr[c + 1]; ++e) {
      const int en = entries_g[e];
      const int j = (en > 0 ? en : -en) - 1;
      ptr[(j / W5) * k + c + 1] += 1u;
    }
  __syncthreads();
  // 2. inclusive scan of ptr[1..nslot] (contiguous segment per thread)
  {
    const int per = (nslot + 511) / 512;
    const int a = 1 + tid * per, b = min(nslot + 1, a + per);
    uint32_t sum = 0u;
    for (int i = a; i < b; ++i) sum += ptr[i];
    uint32_t inc = sum;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, inc, o);
      if (lane >= o) inc += y;
    }
    if (lane == 31) red[warp] = inc;
    __syncthreads();
    if (warp == 0) {
      uint32_t w = lane < 16 ? red[lane] : 0u;
#pragma unroll
      for (int o = 1; o < 16; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, w, o);
        if (lane >= o) w += y;
      }
      if (lane < 16) red[lane] = w;
    }
    __syncthreads();
    uint32_t run = inc - sum + (warp ? red[warp - 1] : 0u);
    for (int i = a; i < b; ++i) {
      run += ptr[i];
      ptr[i] = run;
    }
  }
  __syncthreads();
  // 3. codes in chunk-major order, ascending j inside every (chunk, column):
  // sign in bit 15, byte offset of row (j mod W5) of Xt in bits 0..14
  for (int c = tid; c < k; c += 512) {
    int q = -1;
    uint32_t pos = 0u;
    for (int e = col_ptr[c]; e < col_ptr[c + 1]; ++e) {
      const int en = entries_g[e];
      const int j = (en > 0 ? en : -en) - 1;
      if (j / W5 != q) {
        q = j / W5;
        pos = ptr[q * k + c];
      }
      codes[pos++] = (uint16_t)((en < 0 ? 0x8000 : 0) | ((j % W5) * R5 * 4));
    }
  }
  if (tid == 0) {
    for (int q = 0; q < C::S; ++q) ptx::mbar_init(&full[q], 1);
    ptx::fence_mbar_init();
  }
  const int64_t ntiles = (m + R5 - 1) / R5;
  const int64_t my_tiles = ((int64_t)blockIdx.x < ntiles) ? (ntiles - blockIdx.x + gridDim.x - 1) / gridDim.x : 0;
  const int64_t steps = my_tiles * nch;
  __syncthreads();
  if (steps == 0) return;

  // one thread: step `st` (tile blockIdx.x + (st / nch) gridDim.x, chunk st % nch)
  // into ring stage st % S as NBOX swizzled boxes of 128 rows x 128 bytes
  // (rows past m and columns past n arrive as zeros)
  auto issue = [&](int64_t st) {
    const int r0 = (int)(((int64_t)blockIdx.x + (st / nch) * gridDim.x) * R5);
    const int j0 = (int)((st % nch) * W5);
    const int q = (int)(st % C::S);
    ptx::fence_proxy_async_smem();  // this stage was last read by generic loads
    ptx::mbar_arrive_expect_tx(&full[q], (uint32_t)C::STAGE);
    const uint32_t dst = ptx::smem_u32(ring + (size_t)q * C::STAGE);
#pragma unroll
    for (int b = 0; b < C::NBOX; ++b) ptx::tma_load_2d(dst + b * C::BOX_BYTES, &tmx, j0 + b * C::BOXW, r0, &full[q]);
  };
  if (tid == 0)
    for (int64_t st = 0; st < (steps < C::S ? steps : C::S); ++st) issue(st);

  const int cpw = (k + 15) / 16;
  const int c0 = warp * cpw;
  float acc[8][4];
  uint32_t mxb = 0u;
  float umx = 0.f;
  for (int64_t st = 0; st < steps; ++st) {
    const int q = (int)(st % C::S);
    const int chunk = (int)(st % nch);
    const int64_t r0 = ((int64_t)blockIdx.x + (st / nch) * gridDim.x) * R5;
    const bool ok = ptx::mbar_wait(&full[q], (uint32_t)((st / C::S) & 1), 2000000000ull);
    float* xc = xt + (size_t)(st & 1) * (W5 * R5);
    if (ok) {
      // transpose: item = (row, 16-byte chunk); chunk c of box b, row r sits at
      // b * BOX_BYTES + r * 128 + ((c ^ (r & 7)) << 4) (128-byte swizzle)
      const unsigned char* stage = ring + (size_t)q * C::STAGE;
      const int row = tid % R5;
#pragma unroll
      for (int qq = 0; qq < R5 * C::CHUNKS / 512; ++qq) {
        const int ch = tid / R5 + (512 / R5) * qq;
        const int b = ch / 8, c = ch % 8;
        const uint4 v = *reinterpret_cast<const uint4*>(stage + b * C::BOX_BYTES + row * 128 + ((c ^ (row & 7)) << 4));
        const T* e = reinterpret_cast<const T*>(&v);
        float* dst = xc + ch * C::EPC * R5 + row;
#pragma unroll
        for (int u = 0; u < C::EPC; ++u) {
          const float x = XType<DT>::to_acc(e[u]);
          mxb = max(mxb, __float_as_uint(x) & 0x7fffffffu);
          dst[u * R5] = x;
        }
      }
    }
    if (__syncthreads_or(ok ? 0 : 1)) {
      if (tid == 0) {
        atomicOr(status, ST_TIMEOUT);
        for (int64_t w = st; w < steps && w < st + C::S; ++w)
          ptx::mbar_wait(&full[w % C::S], (uint32_t)((w / C::S) & 1), 100000000ull);
      }
      __syncthreads();
      return;
    }
    if (tid == 0 && st + C::S < steps) issue(st + C::S);

    if (chunk == 0) {
#pragma unroll
      for (int t = 0; t < 8; ++t)
#pragma unroll
        for (int r = 0; r < 4; ++r) acc[t][r] = 0.f;
    }
    const char* xl = reinterpret_cast<const char*>(xc) + lane * 16;
    // begin offsets of the warp's columns in this chunk: lanes 0..cpw load
    // ptr[chunk k + c0 + lane] (the last one is the end of column c0 + cpw - 1)
    const int pi = chunk * k + c0 + lane;
    const uint32_t myp = ptr[pi <= nslot ? pi : nslot];
#pragma unroll
    for (int t = 0; t < 8; ++t) {
      const int c = c0 + t;
      const int b = (int)__shfl_sync(0xffffffffu, myp, t);
      const int e = (int)__shfl_sync(0xffffffffu, myp, t + 1);
      if (t < cpw && c < k) {
        float a0 = acc[t][0], a1 = acc[t][1], a2 = acc[t][2], a3 = acc[t][3];
#pragma unroll 2
        for (int i = b; i < e; ++i) {
          const uint32_t code = codes[i];
          const float4 v = *reinterpret_cast<const float4*>(xl + (code & 0x7fffu));
          const float sg = __uint_as_float(((code & 0x8000u) << 16) | 0x3f800000u);
          a0 = fmaf(sg, v.x, a0);
          a1 = fmaf(sg, v.y, a1);
          a2 = fmaf(sg, v.z, a2);
          a3 = fmaf(sg, v.w, a3);
        }
        acc[t][0] = a0;
        acc[t][1] = a1;
        acc[t][2] = a2;
        acc[t][3] = a3;
      }
    }
    if (chunk == nch - 1) {
      // tile done: rows r0 + 4 lane + i, columns c0 .. c0 + cpw - 1 of U
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const int64_t r = r0 + 4 * lane + i;
        if (r >= m) continue;
        float* dst = U + r * ldu + c0;
        if (vec_u && (cpw & 3) == 0 && c0 + cpw <= k) {
#pragma unroll
          for (int t = 0; t < 8; t += 4)
            if (t < cpw) {
              const float4 v = make_float4(acc[t][i], acc[t + 1][i], acc[t + 2][i], acc[t + 3][i]);
              umx = fmaxf(umx, fmaxf(fmaxf(fabsf(v.x), fabsf(v.y)), fmaxf(fabsf(v.z), fabsf(v.w))));
              *reinterpret_cast<float4*>(dst + t) = v;
            }
        } else {
#pragma unroll
          for (int t = 0; t < 8; ++t)
            if (t < cpw && c0 + t < k) {
              umx = fmaxf(umx, fabsf(acc[t][i]));
              dst[t] = acc[t][i];
            }
        }
      }
    }
  }
  umx = warp_max(umx);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) mxb = max(mxb, __shfl_xor_sync(0xffffffffu, mxb, o));
  if (lane == 0) {
    atomic_max_nonneg(absmax + 1, umx);
    if (mxb >= 0x7f800000u) atomicOr(status, ST_NONFINITE);
    else atomic_max_nonneg(absmax, __uint_as_float(mxb));
  }
}

template <int DT>
static bool sketch_sparse5_dispatch(Launcher& L, const void* X, int64_t m, int64_t n, int64_t ldx, int k,
                                    const int32_t* col_ptr, const int32_t* entries, int32_t* codes_g, float* U,
                                    int64_t ldu, float* absmax, int* status) {
  using C = Sk5<DT>;
  const int64_t nch = (n + W5 - 1) / W5;
  // the (chunk, column) begin offsets live in shared memory
  if (k > 128 || n >= 65536 || m >= ((int64_t)1 << 31) || (int64_t)k * nch + 1 > PTR5) return false;
  CUtensorMap tm;
  const CUtensorMapDataType dt = C::ELEM == 4 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16;
  if (!make_tmap_2d_sw128(&tm, X, dt, C::ELEM, (uint64_t)m, (uint64_t)n, (uint64_t)ldx * C::ELEM, R5, C::BOXW))
    return false;
  cudaFuncSetAttribute(sketch_sparse5_kernel<DT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::SMEM);
  const int64_t ntiles = (m + R5 - 1) / R5;
  const int grid = (int)(ntiles < L.num_sms ? ntiles : L.num_sms);
  const int vec_u = (((uintptr_t)U & 15u) == 0 && (ldu & 3) == 0) ? 1 : 0;
  sketch_sparse5_kernel<DT><<<grid, 512, C::SMEM, L.stream>>>(tm, m, n, k, col_ptr, entries,
                                                              reinterpret_cast<uint16_t*>(codes_g), U, ldu, vec_u,
                                                              absmax, status);
  L.count(1);
  return true;
}

size_t sketch_off_bytes(int64_t n, int k) {
  // worst case over the element types: chunks of 128 columns; plus room for
  // the re-encoded entry codes (n * k int32) of the wide kernel
  return (size_t)k * (size_t)((n + 127) / 128 + 1) * 4 + 256 + (size_t)n * k * 4;
}

static int32_t* codes_area(int32_t* off, int64_t n, int k) {
  const size_t a = ((size_t)k * (size_t)((n + 127) / 128 + 1) * 4 + 255) & ~(size_t)255;
  return reinterpret_cast<int32_t*>(reinterpret_cast<char*>(off) + a);
}

void launch_sketch_sparse(Launcher& L, const void* X, int xt, int64_t m, int64_t n, int64_t ldx, int k,
                          const int32_t* col_ptr, const int32_t* entries, int32_t* off, void* U, int64_t ldu,
                          float* absmax, int* status) {
  switch (xt) {
    case LSPCA_F64:
      sketch_sparse_dispatch<LSPCA_F64>(L, X, m, n, ldx, k, col_ptr, entries, off, U, ldu, absmax, status);
      break;
    case LSPCA_F32:
      if (!sketch_sparse5_dispatch<LSPCA_F32>(L, X, m, n, ldx, k, col_ptr, entries, codes_area(off, n, k),
                                              (float*)U, ldu, absmax, status) &&
          !sketch_sparse4_dispatch<LSPCA_F32>(L, X, m, n, ldx, k, col_ptr, entries, off, codes_area(off, n, k),
                                              (float*)U, ldu, absmax, status))
        sketch_sparse_dispatch<LSPCA_F32>(L, X, m, n, ldx, k, col_ptr, entries, off, U, ldu, absmax, status);
      break;
    case LSPCA_BF16:
      if (!sketch_sparse5_dispatch<LSPCA_BF16>(L, X, m, n, ldx, k, col_ptr, entries, codes_area(off, n, k),
                                               (float*)U, ldu, absmax, status) &&
          !sketch_sparse4_dispatch<LSPCA_BF16>(L, X, m, n, ldx, k, col_ptr, entries, off, codes_area(off, n, k),
                                               (float*)U, ldu, absmax, status))
        sketch_sparse_dispatch<LSPCA_BF16>(L, X, m, n, ldx, k, col_ptr, entries, off, U, ldu, absmax, status);
      break;
    case LSPCA_E4M3:
      if (!sketch_sparse4_dispatch<LSPCA_E4M3>(L, X, m, n, ldx, k, col_ptr, entries, off, codes_area(off, n, k),
                                               (float*)U, ldu, absmax, status))
        sketch_sparse_dispatch<LSPCA_E4M3>(L, X, m, n, ldx, k, col_ptr, entries, off, U, ldu, absmax, status);
      break;
  }
}

// Scan X for NaN/Inf and its largest magnitude (the dense-Omega paths, where the
// sketch runs on tensor cores or as a plain GEMM and does not see every element).
// One warp per row at a time; 16-byte loads when the rows are 16-byte aligned.
template <int DT>
__global__ void scan_x_kernel(const void* __restrict__ Xv, int64_t m, int64_t n, int64_t ldx, float* absmax,
                              int* status) {
  using T = typename XType<DT>::T;
  constexpr int ES = (int)sizeof(T);
  constexpr int EPV = 16 / ES;
  const char* X = reinterpret_cast<const char*>(Xv);
  const int lane = threadIdx.x & 31;
  const int64_t wg = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const bool vec = (((uintptr_t)Xv & 15u) == 0) && ((ldx * ES) % 16 == 0);
  const int64_t nv = vec ? n / EPV : 0;  // full 16-byte vectors per row
  float amax = 0.f;
  bool bad = false;
  auto take = [&](T e) {
    const float v = (float)XType<DT>::to_acc(e);
    if (!isfinite(v)) bad = true;
    amax = fmaxf(amax, fabsf(v));
  };
  for (int64_t r = wg; r < m; r += nw) {
    const char* row = X + r * ldx * ES;
#pragma unroll 4
    for (int64_t v = lane; v < nv; v += 32) {
      const uint4 q = __ldg(reinterpret_cast<const uint4*>(row) + v);
      const T* e = reinterpret_cast<const T*>(&q);
#pragma unroll
      for (int u = 0; u < EPV; ++u) take(e[u]);
    }
    for (int64_t c = nv * EPV + lane; c < n; c += 32) take(reinterpret_cast<const T*>(row)[c]);
  }
  amax = warp_max(amax);
  const unsigned anybad = __ballot_sync(0xffffffffu, bad);
  if (lane == 0) {
    atomic_max_nonneg(absmax, amax);
    if (anybad) atomicOr(status, ST_NONFINITE);
  }
}

void launch_scan_x(Launcher& L, const void* X, int xt, int64_t m, int64_t n, int64_t ldx, float* absmax, int* status) {
  const int threads = 256, blocks = 4 * L.num_sms;
  switch (xt) {
    case LSPCA_F64: scan_x_kernel<LSPCA_F64><<<blocks, threads, 0, L.stream>>>(X, m, n, ldx, absmax, status); break;
    case LSPCA_F32: scan_x_kernel<LSPCA_F32><<<blocks, threads, 0, L.stream>>>(X, m, n, ldx, absmax, status); break;
    case LSPCA_BF16: scan_x_kernel<LSPCA_BF16><<<blocks, threads, 0, L.stream>>>(X, m, n, ldx, absmax, status); break;
    case LSPCA_E4M3: scan_x_kernel<LSPCA_E4M3><<<blocks, threads, 0, L.stream>>>(X, m, n, ldx, absmax, status); break;
  }
  L.count(1);
}

}  // namespace lspca
