// cg_f32.cu -- binary32 instantiation of the persistent CG kernels (Dot2
// compensated dot products, binary64 scalars).
#include "cg_launch.cuh"

namespace lap5 {

size_t ws_bytes_f32(int nx, int ny, int ldw, int variant) {
  (void)nx;
  return ws_bytes_t<float>(ny, ldw, variant);
}

// Lane vector: 8 columns (two 16-byte groups 128 columns apart) halve the
// per-row work of the row march -- ring waits and copy issue, halo and edge
// handling -- per point; narrow grids keep 4 so that strips stay busy.
// Classic CG with the shared-memory ring only: NewCG and the register march
// keep too many rows live for eight columns a lane.
int solve_f32(const SolvePlan& p, cudaStream_t st) {
  if (p.opts.lane_vec == 2) return LAP5CG_ERR_UNSUPPORTED;
  const bool v8_ok = p.variant == LAP5CG_CLASSIC && p.opts.ring_slots >= 0;
  if (p.opts.lane_vec == 8) return v8_ok ? solve_typed<float, 8>(p, st) : LAP5CG_ERR_UNSUPPORTED;
  if (p.opts.lane_vec == 0 && v8_ok && p.nx >= 1024) {
    const int rc = solve_typed<float, 8>(p, st);
    if (rc != LAP5CG_ERR_UNSUPPORTED) return rc;  // units too short for the ring: four columns a lane
  }
  return solve_typed<float, 4>(p, st);
}

}  // namespace lap5
