// Tensor-core passes (placeholder: reports unavailable until the tcgen05 kernels land).
#include "tc.h"

namespace lspca {

bool tc_available() { return false; }
void plan_tc_chain(char*, TcChainWs& w, int, int64_t, int64_t, int, bool, int) { w.bytes = 0; }
void tc_chain_main(Launcher&, const void*, int, int64_t, int64_t, int64_t, const float*, int, TcChainWs&,
                   const float*, bool) {}
void tc_chain_reduce(Launcher&, int64_t, int, TcChainWs&, double*, double*) {}
void tc_sketch_bf16(Launcher&, const void*, int64_t, int64_t, int64_t, const void*, int, float*, float*) {}
void plan_tc_project(char*, TcProjectWs& w, int, int64_t, int) { w.bytes = 0; }
void tc_project(Launcher&, const void*, int, int64_t, int64_t, int64_t, const float*, int, TcProjectWs&, float*) {}

}  // namespace lspca
