// cg_f32.cu -- binary32 instantiation of the persistent CG kernels (Dot2
// compensated dot products, binary64 scalars).
#include "cg_launch.cuh"

namespace lap5 {

size_t ws_bytes_f32(int nx, int ny, int ldw, int variant) {
  (void)nx;
  return ws_bytes_t<float>(ny, ldw, variant);
}

int solve_f32(const SolvePlan& p, cudaStream_t st) { return solve_typed<float, 4>(p, st); }

}  // namespace lap5
