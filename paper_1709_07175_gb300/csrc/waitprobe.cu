// Failure path of the device wait discipline, runnable on purpose without a
// fault.  Every tensor-core pipeline waits on mbarriers with a time limit
// (ptx::mbar_wait): when a phase never completes, the waiting role sets the
// timeout bit of the status word, raises the CTA's abort flag, the other roles
// see the flag and leave their loops, and the kernel ends normally, so the
// context stays usable and the host reads LSPCA_ERR_TIMEOUT.  This kernel runs
// that sequence on a barrier no thread ever arrives at, so tests can check the
// status path and that the next fit on the same context still succeeds.
#include "common.cuh"
#include "kernels.h"
#include "tc_ptx.cuh"

namespace lspca {
namespace {

// warp 0: the waiting role; warps 1-3: roles that poll the abort flag (their
// own loop bounded at twice the limit plus a millisecond).
__global__ void __launch_bounds__(128) wait_probe_kernel(uint64_t limit_ns, int* status, int64_t* waited_ns) {
  __shared__ __align__(8) uint64_t never;  // the barrier whose phase never completes
  __shared__ volatile int abort_flag;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    ptx::mbar_init(&never, 1);
    ptx::fence_mbar_init();
    abort_flag = 0;
  }
  __syncthreads();
  if (warp == 0) {
    if (lane == 0) {
      const uint64_t t0 = ptx::globaltimer();
      const bool ok = ptx::mbar_wait(&never, 0u, limit_ns);
      const uint64_t t1 = ptx::globaltimer();
      if (!ok) {
        atomicOr(status, ST_TIMEOUT);
        __threadfence_block();
        abort_flag = 1;
      }
      if (waited_ns) *waited_ns = (int64_t)(t1 - t0);
    }
    __syncwarp();
  } else {
    const uint64_t t0 = ptx::globaltimer();
    const uint64_t bound = 2 * limit_ns + 1000000ull;
    while (!abort_flag) {
      if (ptx::globaltimer() - t0 > bound) {
        atomicOr(status, ST_TIMEOUT);
        break;
      }
      __nanosleep(1000);
    }
  }
  __syncthreads();
}

}  // namespace

void launch_wait_probe(Launcher& L, uint64_t limit_ns, int* status, int64_t* waited_ns) {
  wait_probe_kernel<<<1, 128, 0, L.stream>>>(limit_ns, status, waited_ns);
  L.count(1);
}

}  // namespace lspca
