// cg_f64.cu -- binary64 instantiation of the persistent CG kernels.
#include "cg_launch.cuh"

namespace lap5 {

size_t ws_bytes_f64(int nx, int ny, int ldw, int variant) {
  (void)nx;
  return ws_bytes_t<double>(ny, ldw, variant);
}

// Lane vector: classic CG with the shared-memory ring runs four columns a lane
// (32 bytes) where the pitches allow it: half the per-row work per point, among
// it the halo column's p = r + beta p, which every lane of the warp executes
// (one FP64 instruction a row, 0.5 a point with two columns).  NewCG, the
// register march and the reproducible mode keep two.
int solve_f64(const SolvePlan& p, cudaStream_t st) {
  const int lv = p.opts.lane_vec;
  if (p.opts.reproducible) return (lv == 0 || lv == 2) ? solve_typed<double, 2, true>(p, st) : LAP5CG_ERR_UNSUPPORTED;
  if (lv == 8) return LAP5CG_ERR_UNSUPPORTED;
  const bool v4_ok = p.variant == LAP5CG_CLASSIC && p.opts.ring_slots >= 0 && p.ld % 4 == 0 && p.ldw % 4 == 0;
  if (lv == 4 && !v4_ok) return LAP5CG_ERR_UNSUPPORTED;
  if ((lv == 4 || lv == 0) && v4_ok) {
    const int rc = solve_typed<double, 4>(p, st);
    if (rc != LAP5CG_ERR_UNSUPPORTED || lv == 4) return rc;  // units too short for the ring: two columns a lane
  }
  return solve_typed<double, 2>(p, st);
}

}  // namespace lap5
