// Tensor-core reduction map Y = X V (Sec. III-B.2: pi(x) = V^T x for every
// row) on sm_103a with tcgen05/TMEM.
//
// GEMM view: M = 128 rows of X per tile, N = k padded to a multiple of 64,
// K = n.  A = the X tile (K-major: rows of X are contiguous in K), B = V
// (MN-major: rows of V are contiguous in N).
//
// Number formats.
// * FP32 X: x s_r = hi + lo with FP16 pieces, where s_r is a power of two
//   chosen per row and per k-step from the row's max |x| in that step (a
//   half-warp reduction over the 64 values the converter already holds), so no
//   extra pass over X is needed; V t = hi + lo likewise with one power of two
//   t from max|V|.  Three products hi*hi + hi*lo + lo*hi.
// * BF16 X: X exact; V split into a BF16 pair; two products.
// * E4M3 X: values widened exactly to BF16; V split as for BF16.
//
// Accumulation.  The tensor core accumulates one k-step (64 columns) per
// segment into TMEM region A (FP32 accumulation into TMEM behaves like
// round-toward-zero on GB300); the epilogue unscales each row of the segment
// by 1 / (s_r t) and folds it into a round-to-nearest FP32 running sum S in
// TMEM region B, then writes S as the rows of Y after the last k-step.
//
// Structure (one persistent CTA per SM, 13 warps, as the pass-F kernel):
// warps 0-7 convert X into the 128B-swizzled K-major A layout (one k-step
// ahead in registers) and warp 0 lane 0 streams the pre-split, pre-swizzled V
// tile of the stage with one cp.async.bulk; warps 8-11 run the epilogue;
// warp 12 allocates TMEM and issues tcgen05.mma.  All waits are bounded.
#include <type_traits>

#include "common.cuh"
#include "tc.h"
#include "tc_ptx.cuh"

namespace lspca {
namespace tcp {

constexpr int BK = 64;
constexpr int CONV_WARPS = 8;
constexpr int CONV_THREADS = 256;
constexpr int EPI_WARP0 = 8;
constexpr int MMA_WARP = 12;
constexpr int THREADS = 13 * 32;
constexpr uint64_t kWaitNs = 2000000000ull;

enum XKind { XK_F32 = 0, XK_BF16 = 1, XK_E4M3 = 2 };

struct Params {
  const void* X;
  int64_t ldx;
  int64_t m, n;
  int k;
  const uint8_t* vt;    // pre-tiled V: per k-step [hi | lo], 256 * NPAD bytes
  const float* vscale;  // device: t (FP32 path) at [0]
  float* Y;             // m x k FP32
  int* status;
  const TcProjUnit* units;  // table mode (serving batches): tiles of many requests
  const int* nunits;        // device count of the table
};

// The tile being processed: from the single matrix, or from the table.
struct TileInfo {
  const void* X;
  int64_t ldx, m, row0, n;
  int k;
  const uint8_t* vt;
  const float* vscale;
  float* Y;
};

__device__ __forceinline__ TileInfo tile_info(const Params& p, int64_t t) {
  TileInfo ti;
  if (p.units) {
    const TcProjUnit& u = p.units[t];
    ti.X = u.X;
    ti.ldx = u.ldx;
    ti.m = u.m;
    ti.row0 = u.row0;
    ti.n = u.n;
    ti.k = u.k;
    ti.vt = u.vt;
    ti.vscale = u.vscale;
    ti.Y = u.Y;
  } else {
    ti.X = p.X;
    ti.ldx = p.ldx;
    ti.m = p.m;
    ti.row0 = t * 128;
    ti.n = p.n;
    ti.k = p.k;
    ti.vt = p.vt;
    ti.vscale = p.vscale;
    ti.Y = p.Y;
  }
  return ti;
}

template <int XK, int NT>
struct Cfg {
  static constexpr int NPAD = 64 * NT;
  static constexpr int PA = (XK == XK_F32) ? 2 : 1;            // A parts
  static constexpr uint32_t A_BYTES = 128 * BK * 2;             // 16 KB
  static constexpr uint32_t B_BYTES = BK * NPAD * 2;            // one part
  static constexpr uint32_t SBO_B = NT * 1024;
  static constexpr uint32_t STAGE_BYTES = 2 * B_BYTES + PA * A_BYTES;
  static constexpr int STAGES = (STAGE_BYTES * 3 <= 200 * 1024) ? 3 : 2;
  static constexpr int RING = STAGES + 2;                      // per-row scale ring
  static constexpr size_t SMEM = 1024 + STAGES * STAGE_BYTES + RING * 128 * 4 + 256 + 8192;
};

__device__ __forceinline__ float pow2_scale_row(float amax) {
  if (!(amax > 0.f) || !isfinite(amax)) return 1.f;
  int e;
  frexpf(amax, &e);
  return ldexpf(1.f, 14 - e);
}

__device__ __forceinline__ uint2 pack_half4(float a, float b, float c, float d) {
  __half2 x = __floats2half2_rn(a, b), y = __floats2half2_rn(c, d);
  return make_uint2(*reinterpret_cast<uint32_t*>(&x), *reinterpret_cast<uint32_t*>(&y));
}

template <int XK, int NT>
__global__ void __launch_bounds__(THREADS, 1) project_kernel(Params p) {
  using C = Cfg<XK, NT>;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  float* scales = reinterpret_cast<float*>(smem + C::STAGES * C::STAGE_BYTES);
  uint64_t* full = reinterpret_cast<uint64_t*>(scales + C::RING * 128);
  uint64_t* empty = full + C::STAGES;
  uint64_t* accf = empty + C::STAGES;
  uint64_t* acce = accf + 1;
  uint64_t* drain = acce + 1;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(drain + 1);
  int* abort_flag = reinterpret_cast<int*>(tmem_slot + 1);

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int64_t tiles = p.units ? (int64_t)*p.nunits : (p.m + 127) / 128;

  if (tid == 0) {
    for (int s = 0; s < C::STAGES; ++s) {
      ptx::mbar_init(&full[s], CONV_WARPS + 1);
      ptx::mbar_init(&empty[s], 1);
    }
    ptx::mbar_init(accf, 1);
    ptx::mbar_init(acce, 4);
    ptx::mbar_init(drain, 1);
    *abort_flag = 0;
    ptx::fence_mbar_init();
  }
  if (warp == MMA_WARP) ptx::tmem_alloc(tmem_slot, 512);
  ptx::tc_fence_before();
  __syncthreads();
  ptx::tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  const uint32_t sbase = ptx::smem_u32(smem);
  auto fail = [&]() {
    atomicOr(p.status, ST_TIMEOUT);
    atomicExch(abort_flag, 1);
  };
  auto aborted = [&]() { return *(volatile int*)abort_flag != 0; };

  if (warp < CONV_WARPS) {
    // ------------------------------------------------------------ converters
    constexpr int NV = (XK == XK_F32) ? 8 : (XK == XK_BF16 ? 4 : 2);  // 16-byte vectors per thread per k-step
    auto load = [&](const TileInfo& ti, int ks, uint4 (&dst)[NV]) {
#pragma unroll
      for (int q = 0; q < NV; ++q) {
        const int f = tid + CONV_THREADS * q;
        int row, col;
        if (XK == XK_F32) { row = f / 16; col = (f % 16) * 4; }
        else if (XK == XK_BF16) { row = f / 8; col = (f % 8) * 8; }
        else { row = f / 4; col = (f % 4) * 16; }
        const int64_t gr = ti.row0 + row, gc = (int64_t)ks * BK + col;
        if (gr < ti.m && gc < ti.n) {
          const char* src = (const char*)ti.X + (gr * ti.ldx + gc) * (XK == XK_F32 ? 4 : (XK == XK_BF16 ? 2 : 1));
          asm volatile("ld.global.nc.L1::no_allocate.v4.u32 {%0, %1, %2, %3}, [%4];"
                       : "=r"(dst[q].x), "=r"(dst[q].y), "=r"(dst[q].z), "=r"(dst[q].w)
                       : "l"(src));
        } else {
          dst[q] = make_uint4(0u, 0u, 0u, 0u);
        }
      }
    };
    auto store = [&](const uint4 (&r)[NV], uint32_t st, int slot, int ks, int64_t ncols) {
      const uint32_t a_hi = st + 2 * C::B_BYTES, a_lo = a_hi + C::A_BYTES;
#pragma unroll
      for (int q = 0; q < NV; ++q) {
        const int f = tid + CONV_THREADS * q;
        if (XK == XK_F32) {
          const int row = f / 16, col = (f % 16) * 4;
          float v[4] = {__uint_as_float(r[q].x), __uint_as_float(r[q].y), __uint_as_float(r[q].z),
                        __uint_as_float(r[q].w)};
          // zero the tail of a row that ends inside this vector
          const int64_t gc = (int64_t)ks * BK + col;
#pragma unroll
          for (int u = 0; u < 4; ++u)
            if (gc + u >= ncols) v[u] = 0.f;
          float mx = fmaxf(fmaxf(fabsf(v[0]), fabsf(v[1])), fmaxf(fabsf(v[2]), fabsf(v[3])));
#pragma unroll
          for (int o = 1; o < 16; o <<= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
          const float s = pow2_scale_row(mx);
          if ((f % 16) == 0) scales[slot * 128 + row] = s;
          float hi[4], lo[4];
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            const float xs = v[u] * s;
            hi[u] = __half2float(__float2half_rn(xs));
            lo[u] = xs - hi[u];
          }
          const uint32_t off = ptx::k_sw128_offset(row, col);
          const uint2 h = pack_half4(hi[0], hi[1], hi[2], hi[3]);
          const uint2 l = pack_half4(lo[0], lo[1], lo[2], lo[3]);
          asm volatile("st.shared.v2.b32 [%0], {%1, %2};" ::"r"(a_hi + off), "r"(h.x), "r"(h.y) : "memory");
          asm volatile("st.shared.v2.b32 [%0], {%1, %2};" ::"r"(a_lo + off), "r"(l.x), "r"(l.y) : "memory");
        } else if (XK == XK_BF16) {
          const int row = f / 8, col = (f % 8) * 8;
          uint4 v = r[q];
          const int64_t gc = (int64_t)ks * BK + col;
          if (gc + 8 > ncols) {
            uint16_t* e = reinterpret_cast<uint16_t*>(&v);
#pragma unroll
            for (int u = 0; u < 8; ++u)
              if (gc + u >= ncols) e[u] = 0;
          }
          asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(a_hi + ptx::k_sw128_offset(row, col)),
                       "r"(v.x), "r"(v.y), "r"(v.z), "r"(v.w)
                       : "memory");
        } else {
          const int row = f / 4, col = (f % 4) * 16;
          const int64_t gc = (int64_t)ks * BK + col;
          const __nv_fp8_e4m3* e8 = reinterpret_cast<const __nv_fp8_e4m3*>(&r[q]);
          uint32_t w[8];
#pragma unroll
          for (int u = 0; u < 8; ++u) {
            float a = (gc + 2 * u < ncols) ? float(e8[2 * u]) : 0.f;
            float b = (gc + 2 * u + 1 < ncols) ? float(e8[2 * u + 1]) : 0.f;
            __nv_bfloat162 h2 = __floats2bfloat162_rn(a, b);
            w[u] = *reinterpret_cast<uint32_t*>(&h2);
          }
          asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(a_hi + ptx::k_sw128_offset(row, col)),
                       "r"(w[0]), "r"(w[1]), "r"(w[2]), "r"(w[3])
                       : "memory");
          asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(a_hi + ptx::k_sw128_offset(row, col + 8)),
                       "r"(w[4]), "r"(w[5]), "r"(w[6]), "r"(w[7])
                       : "memory");
        }
      }
    };
    // Two register buffers in ping-pong: the loads of step t + 1 are issued
    // before step t is converted and consumed one full iteration later (a
    // register copy from a prefetch buffer would wait for them at once).
    uint4 ra[NV], rb[NV];
    int64_t tile = blockIdx.x;
    int ks = 0;
    int64_t step = 0;
    TileInfo ti, tn;
    auto body = [&](const uint4 (&cur)[NV], uint4 (&nxt)[NV]) -> bool {
      const int nks = (int)((ti.n + BK - 1) / BK);
      int64_t ntile = tile;
      int nks_next = ks + 1;
      if (nks_next >= nks) {
        nks_next = 0;
        ntile += gridDim.x;
      }
      const bool more = ntile < tiles;
      if (more) {
        if (ntile != tile) tn = tile_info(p, ntile);
        load(ntile != tile ? tn : ti, nks_next, nxt);
      }
      const int s = (int)(step % C::STAGES);
      const uint32_t ph = (uint32_t)((step / C::STAGES) & 1);
      if (!ptx::mbar_wait(&empty[s], ph ^ 1u, kWaitNs)) {
        fail();
        return false;
      }
      if (aborted()) return false;
      const uint32_t st = sbase + s * C::STAGE_BYTES;
      if (warp == 0 && lane == 0) {
        ptx::mbar_arrive_expect_tx(&full[s], 2 * C::B_BYTES);
        ptx::bulk_g2s(st, ti.vt + (size_t)ks * 2 * C::B_BYTES, 2 * C::B_BYTES, &full[s]);
      }
      store(cur, st, (int)(step % C::RING), ks, ti.n);
      ptx::fence_proxy_async_smem();
      __syncwarp();
      if (lane == 0) ptx::mbar_arrive(&full[s]);
      ++step;
      if (!more) return false;
      if (ntile != tile) ti = tn;
      tile = ntile;
      ks = nks_next;
      return true;
    };
    if (tile < tiles) {
      ti = tile_info(p, tile);
      tn = ti;
      load(ti, ks, ra);
      while (body(ra, rb) && body(rb, ra)) {
      }
    }
  } else if (warp == MMA_WARP) {
    // ------------------------------------------------------------ MMA issuer
    if (lane == 0) {
      constexpr uint32_t idesc = ptx::idesc_f16(XK == XK_F32 ? 0 : 1, 128, C::NPAD, 0, 1);
      int64_t step = 0;
      bool ok = true;
      for (int64_t tile = blockIdx.x; tile < tiles && ok; tile += gridDim.x) {
        const int nks = (int)((tile_info(p, tile).n + BK - 1) / BK);
        for (int ks = 0; ks < nks; ++ks, ++step) {
          if (!ptx::mbar_wait(acce, (uint32_t)((step & 1) ^ 1), kWaitNs)) {
            fail();
            ok = false;
            break;
          }
          ptx::tc_fence_after();
          const int s = (int)(step % C::STAGES);
          const uint32_t ph = (uint32_t)((step / C::STAGES) & 1);
          if (!ptx::mbar_wait(&full[s], ph, kWaitNs) || aborted()) {
            if (!aborted()) fail();
            ok = false;
            break;
          }
          ptx::tc_fence_after();
          const uint32_t st = sbase + s * C::STAGE_BYTES;
          const uint32_t b_hi = st, b_lo = st + C::B_BYTES, a_hi = st + 2 * C::B_BYTES, a_lo = a_hi + C::A_BYTES;
#pragma unroll
          for (int kk = 0; kk < BK / 16; ++kk) {
            const uint64_t adh = ptx::desc_sw128(a_hi + kk * 32, 16, 1024);
            const uint64_t bdh = ptx::desc_sw128(b_hi + kk * 2 * C::SBO_B, 1024, C::SBO_B);
            const uint64_t bdl = ptx::desc_sw128(b_lo + kk * 2 * C::SBO_B, 1024, C::SBO_B);
            ptx::mma_f16(tmem, adh, bdh, idesc, kk > 0 ? 1u : 0u);
            ptx::mma_f16(tmem, adh, bdl, idesc, 1u);
            if (XK == XK_F32) {
              const uint64_t adl = ptx::desc_sw128(a_lo + kk * 32, 16, 1024);
              ptx::mma_f16(tmem, adl, bdh, idesc, 1u);
            }
          }
          ptx::mma_commit(&empty[s]);
          ptx::mma_commit(accf);
        }
      }
      ptx::mma_commit(drain);
      if (!ptx::mbar_wait(drain, 0u, kWaitNs)) atomicOr(p.status, ST_TIMEOUT);
    }
    __syncwarp();
  } else {
    // ------------------------------------------------------------ epilogue
    const int e = warp - EPI_WARP0;
    const uint32_t lane_base = (uint32_t)(32 * e) << 16;
    int64_t step = 0;
    bool ok = true;
    for (int64_t tile = blockIdx.x; tile < tiles && ok; tile += gridDim.x) {
      const TileInfo ti = tile_info(p, tile);
      const float inv_t = (XK == XK_F32) ? 1.f / *ti.vscale : 1.f;
      const int nks = (int)((ti.n + BK - 1) / BK);
      const int row = 32 * e + lane;
      const int64_t grow = ti.row0 + row;
      for (int ks = 0; ks < nks; ++ks, ++step) {
        if (!ptx::mbar_wait(accf, (uint32_t)(step & 1), kWaitNs) || aborted()) {
          if (!aborted()) fail();
          ok = false;
          break;
        }
        ptx::tc_fence_after();
        const float us = (XK == XK_F32) ? inv_t / scales[(int)(step % C::RING) * 128 + row] : 1.f;
        const bool first = ks == 0, last = ks == nks - 1;
#pragma unroll 1
        for (int c0 = 0; c0 < C::NPAD; c0 += 32) {
          uint32_t a[32], sacc[32];
          ptx::tmem_ld32(tmem + lane_base + (uint32_t)c0, a);
          if (first) {
#pragma unroll
            for (int q = 0; q < 32; ++q) sacc[q] = __float_as_uint(__uint_as_float(a[q]) * us);
          } else {
            ptx::tmem_ld32(tmem + lane_base + (uint32_t)(C::NPAD + c0), sacc);
#pragma unroll
            for (int q = 0; q < 32; ++q)
              sacc[q] = __float_as_uint(fmaf(__uint_as_float(a[q]), us, __uint_as_float(sacc[q])));
          }
          if (!last) {
            ptx::tmem_st32(tmem + lane_base + (uint32_t)(C::NPAD + c0), sacc);
          } else if (grow < ti.m) {
            float* dst = ti.Y + grow * ti.k + c0;
            if (c0 + 32 <= ti.k && (ti.k % 4) == 0) {
#pragma unroll
              for (int q = 0; q < 32; q += 4)
                *reinterpret_cast<float4*>(dst + q) = make_float4(__uint_as_float(sacc[q]), __uint_as_float(sacc[q + 1]),
                                                                  __uint_as_float(sacc[q + 2]),
                                                                  __uint_as_float(sacc[q + 3]));
            } else {
#pragma unroll
              for (int q = 0; q < 32; ++q)
                if (c0 + q < ti.k) dst[q] = __uint_as_float(sacc[q]);
            }
          }
        }
        ptx::tc_fence_before();
        __syncwarp();
        if (lane == 0) ptx::mbar_arrive(acce);
      }
    }
  }
  __syncthreads();
  if (warp == MMA_WARP) {
    ptx::tc_fence_after();
    ptx::tmem_dealloc(tmem, 512);
  }
}

// V (n x k FP32) -> per k-step tiles [hi | lo] in the MN-major SW128 layout
// (8 K-rows x 64 N-columns per 1024-byte atom, N-atoms adjacent), zero padded
// to NPAD columns and to whole k-steps.  FP32 path: FP16 pair of V * t with t
// a power of two from max|V| (vscale[0] = t); else a BF16 pair of V.
__global__ void tile_v_kernel(const float* __restrict__ V, int64_t n, int k, int npad, int f16, const float* amax,
                              float* vscale, uint8_t* __restrict__ out) {
  const int nt = npad / 64;
  const int nks = (int)((n + BK - 1) / BK);
  const uint32_t sbo = nt * 1024;
  const size_t part = (size_t)BK * npad * 2;
  float t = 1.f;
  if (f16) {
    t = pow2_scale_row(*amax);
    if (blockIdx.x == 0 && threadIdx.x == 0) *vscale = t;
  }
  const int64_t total = (int64_t)nks * BK * npad;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int c = (int)(e % npad);
    const int64_t j = e / npad;  // global row of V
    const int ks = (int)(j / BK), kr = (int)(j % BK);
    const float v = (j < n && c < k) ? V[j * k + c] : 0.f;
    uint16_t hb, lb;
    if (f16) {
      const __half h = __float2half_rn(v * t);
      const __half l = __float2half_rn(v * t - __half2float(h));
      hb = *reinterpret_cast<const uint16_t*>(&h);
      lb = *reinterpret_cast<const uint16_t*>(&l);
    } else {
      const __nv_bfloat16 h = __float2bfloat16_rn(v);
      const __nv_bfloat16 l = __float2bfloat16_rn(v - __bfloat162float(h));
      hb = *reinterpret_cast<const uint16_t*>(&h);
      lb = *reinterpret_cast<const uint16_t*>(&l);
    }
    uint8_t* base = out + (size_t)ks * 2 * part;
    const uint32_t off = ptx::mn_sw128_offset(kr, c, sbo);
    *reinterpret_cast<uint16_t*>(base + off) = hb;
    *reinterpret_cast<uint16_t*>(base + part + off) = lb;
  }
}

template <int XK, int NT>
static void launch_project(Launcher& L, const Params& p, int max_tiles) {
  using C = Cfg<XK, NT>;
  cudaFuncSetAttribute(project_kernel<XK, NT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::SMEM);
  const int64_t tiles = p.units ? max_tiles : (p.m + 127) / 128;
  const int grid = (int)(tiles < L.num_sms ? (tiles > 0 ? tiles : 1) : L.num_sms);
  project_kernel<XK, NT><<<grid, THREADS, C::SMEM, L.stream>>>(p);
  L.count(1);
}

template <int XK>
static void launch_project_nt(Launcher& L, const Params& p, int nt, int max_tiles) {
  switch (nt) {
    case 1: launch_project<XK, 1>(L, p, max_tiles); break;
    case 2: launch_project<XK, 2>(L, p, max_tiles); break;
    case 3: launch_project<XK, 3>(L, p, max_tiles); break;
    default: launch_project<XK, 4>(L, p, max_tiles); break;
  }
}

}  // namespace tcp

void plan_tc_project(char* base, TcProjectWs& w, int xt, int64_t n, int k) {
  const int npad = (k + 63) / 64 * 64;
  const int64_t nks = (n + tcp::BK - 1) / tcp::BK;
  size_t off = 0;
  auto take = [&](size_t b) {
    off = (off + 255) & ~(size_t)255;
    char* r = base ? base + off : nullptr;
    off += b;
    return r;
  };
  w.vhi = take((size_t)nks * 2 * tcp::BK * npad * 2);
  w.vlo = take(256);  // scalars: [0] max|V|, [1] t
  w.bytes = off + 256;
  (void)xt;
}

void tc_project(Launcher& L, const void* X, int xt, int64_t m, int64_t n, int64_t ldx, const float* V, int k,
                TcProjectWs& w, float* Y, int* status) {
  const int npad = (k + 63) / 64 * 64;
  float* scal = (float*)w.vlo;
  const bool f16 = xt == LSPCA_F32;
  cudaMemsetAsync(scal, 0, 8, L.stream);
  if (f16) launch_scan_x(L, V, LSPCA_F32, n, k, k, scal, status);
  {
    const int64_t nks = (n + tcp::BK - 1) / tcp::BK;
    const int64_t total = nks * tcp::BK * npad;
    int blocks = (int)((total + 255) / 256);
    if (blocks > 16 * L.num_sms) blocks = 16 * L.num_sms;
    tcp::tile_v_kernel<<<blocks, 256, 0, L.stream>>>(V, n, k, npad, f16 ? 1 : 0, scal, scal + 1, (uint8_t*)w.vhi);
    L.count(1);
  }
  tcp::Params p{};
  p.X = X;
  p.ldx = ldx;
  p.m = m;
  p.n = n;
  p.k = k;
  p.vt = (const uint8_t*)w.vhi;
  p.vscale = scal + 1;
  p.Y = Y;
  p.status = status;
  p.units = nullptr;
  p.nunits = nullptr;
  const int nt = npad / 64;
  if (xt == LSPCA_F32) tcp::launch_project_nt<tcp::XK_F32>(L, p, nt, 0);
  else if (xt == LSPCA_BF16) tcp::launch_project_nt<tcp::XK_BF16>(L, p, nt, 0);
  else tcp::launch_project_nt<tcp::XK_E4M3>(L, p, nt, 0);
}

void tc_project_pretiled(Launcher& L, const void* X, int xt, int64_t m, int64_t n, int64_t ldx, const void* tiles,
                         const float* vscale, int k, float* Y, int* status) {
  tcp::Params p{};
  p.X = X;
  p.ldx = ldx;
  p.m = m;
  p.n = n;
  p.k = k;
  p.vt = (const uint8_t*)tiles;
  p.vscale = vscale;
  p.Y = Y;
  p.status = status;
  p.units = nullptr;
  p.nunits = nullptr;
  const int nt = (k + 63) / 64;
  if (xt == LSPCA_F32) tcp::launch_project_nt<tcp::XK_F32>(L, p, nt, 0);
  else if (xt == LSPCA_BF16) tcp::launch_project_nt<tcp::XK_BF16>(L, p, nt, 0);
  else tcp::launch_project_nt<tcp::XK_E4M3>(L, p, nt, 0);
}

size_t tc_tile_v_bytes(int64_t n, int k) {
  const int npad = (k + 63) / 64 * 64;
  return (size_t)((n + tcp::BK - 1) / tcp::BK) * 2 * tcp::BK * npad * 2;
}

void tc_tile_v(Launcher& L, int xt, const float* V, int64_t n, int k, void* tiles, float* scal, int* status) {
  const int npad = (k + 63) / 64 * 64;
  const bool f16 = xt == LSPCA_F32;
  cudaMemsetAsync(scal, 0, 8, L.stream);
  if (f16) launch_scan_x(L, V, LSPCA_F32, n, k, k, scal, status);
  const int64_t nks = (n + tcp::BK - 1) / tcp::BK;
  const int64_t total = nks * tcp::BK * npad;
  int blocks = (int)((total + 255) / 256);
  if (blocks > 16 * L.num_sms) blocks = 16 * L.num_sms;
  tcp::tile_v_kernel<<<blocks, 256, 0, L.stream>>>(V, n, k, npad, f16 ? 1 : 0, scal, scal + 1, (uint8_t*)tiles);
  L.count(1);
}

void tc_project_batch(Launcher& L, int xt, int k, const TcProjUnit* d_units, const int* d_count, int max_tiles,
                      int* status) {
  tcp::Params p{};
  p.units = d_units;
  p.nunits = d_count;
  p.status = status;
  const int nt = (k + 63) / 64;
  if (xt == LSPCA_F32) tcp::launch_project_nt<tcp::XK_F32>(L, p, nt, max_tiles);
  else if (xt == LSPCA_BF16) tcp::launch_project_nt<tcp::XK_BF16>(L, p, nt, max_tiles);
  else tcp::launch_project_nt<tcp::XK_E4M3>(L, p, nt, max_tiles);
}

}  // namespace lspca
