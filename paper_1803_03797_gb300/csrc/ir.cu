// ir.cu -- FP64 iterative refinement around a binary32 / bf16-p,r inner CG.
#include "launch.h"

namespace lap5 {

size_t ws_bytes_ir(int nx, int ny, int variant, int precision) {
  (void)nx; (void)ny; (void)variant; (void)precision;
  return 0;
}

int solve_ir(const SolvePlan& p, cudaStream_t st) {
  (void)p; (void)st;
  return LAP5CG_ERR_UNSUPPORTED;
}

}  // namespace lap5
