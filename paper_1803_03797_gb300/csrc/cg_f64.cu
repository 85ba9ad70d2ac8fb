// cg_f64.cu -- binary64 instantiation of the persistent CG kernels.
#include "cg_launch.cuh"

namespace lap5 {

size_t ws_bytes_f64(int nx, int ny, int ldw, int variant) {
  (void)nx;
  return ws_bytes_t<double>(ny, ldw, variant);
}

int solve_f64(const SolvePlan& p, cudaStream_t st) {
  if (p.opts.reproducible) return solve_typed<double, 2, true>(p, st);
  return solve_typed<double, 2>(p, st);
}

}  // namespace lap5
