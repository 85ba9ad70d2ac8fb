// ir.cu -- host launch of the mixed-precision kernels: FP64 iterative
// refinement around an inner classic CG stored in binary32 (IR_F32) or with
// bf16 p and r (IR_BF16PR).
#include "ir_kernels.cuh"
#include "cg_launch.cuh"

namespace lap5 {

// Outer (binary64) passes move two columns a lane: their b, x and field rows
// then fit the register budget that the inner passes need.
constexpr int kOuterVec = 2;

template <class TR, int V, bool R>
__global__ void __launch_bounds__(512) k_ir(const IrArgs<TR> a) {
  __shared__ double red[kRedDoubles];
  extern __shared__ __align__(128) unsigned char dsm[];
  GridTeam tm{a.c.ctl, a.c.timeout_ns, 0ull};
  ir_solve<TR, V, kOuterVec, R>(a, tm, red, dsm);
}

static int inner_ld(int nx) { return (nx + 7) / 8 * 8; }

template <class TR>
static size_t ws_ir_t(int nx, int ny) {
  const size_t ldi = (size_t)inner_ld(nx);
  return kCtlBytes + 3 * align_up((size_t)ny * ldi * sizeof(TR), kAlign) + 2 * align_up((size_t)ny * ldi * 4, kAlign);
}

size_t ws_bytes_ir(int nx, int ny, int variant, int precision) {
  if (variant != LAP5CG_CLASSIC) return 0;  // the inner solver is Algorithm 1
  if (precision == LAP5CG_PREC_IR_F32) return ws_ir_t<float>(nx, ny);
  if (precision == LAP5CG_PREC_IR_BF16PR) return ws_ir_t<bf16s>(nx, ny);
  return 0;
}

template <class TR, int V>
static int solve_ir_t(const SolvePlan& p, cudaStream_t st) {
  const int ldi = inner_ld(p.nx);
  const size_t vr = align_up((size_t)p.ny * ldi * sizeof(TR), kAlign);
  const size_t vf = align_up((size_t)p.ny * ldi * 4, kAlign);
  unsigned char* base = p.ws + kCtlBytes;
  if (cudaMemsetAsync(p.ws, 0, 256, st) != cudaSuccess) return LAP5CG_ERR_CUDA;
  LaunchCfg cfg;
  RingGeom rg;
  size_t dyn = 0;
  bool ring = false;
  int rc = pick_ring(reinterpret_cast<const void*>(&k_ir<TR, V, true>), ring_slot_ir(V, (int)sizeof(TR)), p.opts,
                     &rg, &dyn, &ring);
  if (rc != LAP5CG_OK) return rc;
  const void* fn = reinterpret_cast<const void*>(&k_ir<TR, V, true>);
  if constexpr (Lanes<V>::G > 1) {  // eight columns a lane exist with the ring only
    if (!ring) return LAP5CG_ERR_UNSUPPORTED;
  } else if (!ring) {
    fn = reinterpret_cast<const void*>(&k_ir<TR, V, false>);
  }
  rc = plan_units(fn, p.nx, p.ny, V, p.opts, dyn, &cfg);
  if (rc != LAP5CG_OK) return rc;
  if (ring && p.opts.ring_slots == 0 && cfg.seg_rows < kRingMinRows) {  // short units: register march
    if constexpr (Lanes<V>::G > 1) {
      return LAP5CG_ERR_UNSUPPORTED;  // the caller narrows the lane vector
    } else {
      ring = false;
      rg.S = 0;
      dyn = 0;
      fn = reinterpret_cast<const void*>(&k_ir<TR, V, false>);
      rc = plan_units(fn, p.nx, p.ny, V, p.opts, dyn, &cfg);
      if (rc != LAP5CG_OK) return rc;
    }
  }
  IrArgs<TR> a;
  a.c = make_common(p, cfg, rg);
  a.uo = make_units(p.nx, p.ny, kOuterVec, (long long)cfg.ctas * (cfg.threads / 32),
                    p.opts.min_rows > 0 ? p.opts.min_rows : kDefaultMinRows);
  a.b = Grid<const double>{static_cast<const double*>(p.b), p.ld};
  a.x = Grid<double>{static_cast<double*>(p.x), p.ld};
  a.r = Grid<TR>{reinterpret_cast<TR*>(base), ldi};
  a.p0 = Grid<TR>{reinterpret_cast<TR*>(base + vr), ldi};
  a.p1 = Grid<TR>{reinterpret_cast<TR*>(base + 2 * vr), ldi};
  a.z = Grid<float>{reinterpret_cast<float*>(base + 3 * vr), ldi};
  a.d = Grid<float>{reinterpret_cast<float*>(base + 3 * vr + vf), ldi};
  a.store_z = p.opts.store_z > 0 ? 1 : 0;  // binary32 inner passes are bandwidth bound: recompute A p
  a.max_outer = p.opts.max_outer > 0 ? p.opts.max_outer : 60;
  // inner cap: binary32 4 (nx + ny) + 50; bf16 p, r 2 (nx + ny) + 50, the measured
  // best for time to 1e-10 at 4096^2 (5.3 s against 6.3 s with nx + ny + 50;
  // at 8192^2 every cap from 4096 to 65586 converges, in 72 to 89 s)
  a.maxit_inner = p.opts.maxit_inner > 0 ? p.opts.maxit_inner
                                         : (sizeof(TR) == 2 ? 2 * (p.nx + p.ny) + 50 : 4 * (p.nx + p.ny) + 50);
  a.tol_inner = p.opts.tol_inner > 0.0 ? p.opts.tol_inner : (sizeof(TR) == 2 ? 1e-2 : 1e-4);
  void* args[] = {&a};
  return cooperative_launch(fn, cfg, args, st, rg);
}

// Inner lane vector: eight columns (ring kernel) on wide grids, as for the
// binary32 solve; four with the register march.
template <class TR>
static int solve_ir_lanes(const SolvePlan& p, cudaStream_t st) {
  if (p.opts.lane_vec == 2) return LAP5CG_ERR_UNSUPPORTED;
  const bool v8_ok = p.opts.ring_slots >= 0 && p.opts.store_z <= 0;
  if (p.opts.lane_vec == 8) return v8_ok ? solve_ir_t<TR, 8>(p, st) : LAP5CG_ERR_UNSUPPORTED;
  if (p.opts.lane_vec == 0 && v8_ok && p.nx >= 1024) {
    const int rc = solve_ir_t<TR, 8>(p, st);
    if (rc != LAP5CG_ERR_UNSUPPORTED) return rc;
  }
  return solve_ir_t<TR, 4>(p, st);
}

int solve_ir(const SolvePlan& p, cudaStream_t st) {
  if (p.variant != LAP5CG_CLASSIC) return LAP5CG_ERR_UNSUPPORTED;
  if (p.precision == LAP5CG_PREC_IR_F32) return solve_ir_lanes<float>(p, st);
  if (p.precision == LAP5CG_PREC_IR_BF16PR) return solve_ir_lanes<bf16s>(p, st);
  return LAP5CG_ERR_INVALID_ARG;
}

}  // namespace lap5
