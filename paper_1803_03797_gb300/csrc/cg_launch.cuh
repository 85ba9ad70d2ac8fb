// cg_launch.cuh -- host launch of the persistent classic / NewCG kernels for
// one storage type.  Included by cg_f64.cu and cg_f32.cu.
#pragma once

#include "cg_kernels.cuh"
#include "launch.h"

namespace lap5 {

// R: rows staged through the shared-memory ring (bulk asynchronous copies)
// or loaded straight into registers.
// EX: reproducible dot products (exact accumulation; the CTA's accumulators
// live in static shared memory and start at zero).
template <bool EX> struct ExactSmem {
  __device__ __forceinline__ void attach(GridTeam&) {}
};
template <> struct ExactSmem<true> {
  __device__ __forceinline__ void attach(GridTeam& tm) {
    __shared__ unsigned long long xs[kExactSlots * kExactLimbs];
    __shared__ unsigned xsb[kExactSlots];
    for (int t = threadIdx.x; t < kExactSlots * kExactLimbs; t += blockDim.x) xs[t] = 0ull;
    if (threadIdx.x < kExactSlots) xsb[threadIdx.x] = 0u;
    __syncthreads();
    tm.xs = xs;
    tm.xsb = xsb;
  }
};

template <class T, int V, bool R, bool EX = false>
__global__ void __launch_bounds__(512) k_classic(const ClassicArgs<T> a) {
  __shared__ double red[kRedDoubles];
  extern __shared__ __align__(128) unsigned char dsm[];
  GridTeam tm{a.c.ctl, a.c.timeout_ns, 0ull};
  ExactSmem<EX>().attach(tm);
  classic_solve<T, V, R, EX>(a, tm, red, dsm);
}

// ST: the stabilised alpha (plain dot products only)
template <class T, int V, bool R, bool EX = false, bool ST = false>
__global__ void __launch_bounds__(512) k_newcg(const NewcgArgs<T> a) {
  __shared__ double red[kRedDoubles];
  extern __shared__ __align__(128) unsigned char dsm[];
  GridTeam tm{a.c.ctl, a.c.timeout_ns, 0ull};
  ExactSmem<EX>().attach(tm);
  newcg_solve<T, V, R, EX, ST>(a, tm, red, dsm);
}

// Ring geometry for a kernel pair: tries the ring kernel first; falls back to
// the register kernel when the ring is off or does not fit.
inline int pick_ring(const void* fn_ring, int slot_bytes, const lap5cg_opts& o, RingGeom* rg, size_t* dyn,
                     bool* use_ring, bool auto_on = true) {
  int rc = choose_ring(fn_ring, slot_bytes, o, warps_of(o), rg, dyn, auto_on);
  if (rc != LAP5CG_OK) return rc;
  *use_ring = rg->S > 0;
  return LAP5CG_OK;
}

template <class T>
inline size_t ws_bytes_t(int ny, int ldw, int variant) {
  const size_t vec = align_up((size_t)ny * (size_t)ldw * sizeof(T), kAlign);
  const int nvec = (variant == LAP5CG_NEWCG) ? 6 : 4;
  return kCtlBytes + nvec * vec;
}

inline int cooperative_launch(const void* func, const LaunchCfg& cfg, void** args, cudaStream_t st,
                              const RingGeom& rg) {
  // every warp's ring must lie inside the CTA's dynamic shared memory
  if (rg.S > 0 && cfg.dyn_smem < (size_t)(cfg.threads / 32) * (size_t)rg.warp_bytes) return LAP5CG_ERR_INVALID_ARG;
  cudaLaunchConfig_t lc = {};
  lc.gridDim = dim3(cfg.ctas);
  lc.blockDim = dim3(cfg.threads);
  lc.dynamicSmemBytes = cfg.dyn_smem;
  lc.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  lc.attrs = attr;
  lc.numAttrs = 1;
  cudaError_t e = cudaLaunchKernelExC(&lc, func, args);
  return e == cudaSuccess ? LAP5CG_OK : LAP5CG_ERR_CUDA;
}

inline SolveCommon make_common(const SolvePlan& p, const LaunchCfg& cfg, const RingGeom& rg) {
  SolveCommon c;
  c.nx = p.nx;
  c.ny = p.ny;
  c.un.ns = cfg.ns;
  c.un.nseg = cfg.nseg;
  c.un.seg_rows = cfg.seg_rows;
  c.un.nunits = cfg.nunits;
  c.ctl = reinterpret_cast<Ctl*>(p.ws);
  c.info = p.info;
  c.history = p.opts.history;
  c.tol = p.tol;
  c.maxit = p.maxit;
  c.true_res = p.opts.true_residual;
  const double to = p.opts.timeout_s > 0.0 ? p.opts.timeout_s : 2.0;
  c.timeout_ns = (long long)(to * 1e9);
  c.rg = rg;
  c.err = &c.ctl->status;
  c.abort_flag = &c.ctl->abort;
  return c;
}

// Lane vectors that exist with the shared-memory ring only: eight columns (two
// groups), and four binary64 columns (32 bytes a lane: the register march
// would keep too many rows live).  NewCG runs neither: it keeps six vectors live.
template <class T, int V>
struct RingOnly {
  static constexpr bool value = Lanes<V>::G > 1 || (sizeof(T) == 8 && V == 4);
};

// EX: reproducible dot products.  Their units start at multiples of 16 rows
// and the first of the control block's three exact accumulators starts at zero.
template <class T, int V, bool EX = false>
int solve_typed(const SolvePlan& p, cudaStream_t st) {
  const size_t vec = align_up((size_t)p.ny * (size_t)p.ldw * sizeof(T), kAlign);
  unsigned char* base = p.ws + kCtlBytes;
  auto vecp = [&](int k) { return reinterpret_cast<T*>(base + (size_t)k * vec); };
  const size_t ctl_zero = EX ? offsetof(Ctl, part) : 256;
  if (cudaMemsetAsync(p.ws, 0, ctl_zero, st) != cudaSuccess) return LAP5CG_ERR_CUDA;
  const int row_align = EX ? kExactRows : 1;
  LaunchCfg cfg;
  if (p.variant == LAP5CG_CLASSIC) {
    RingGeom rg;
    size_t dyn = 0;
    bool ring = false;
    int rc = pick_ring(reinterpret_cast<const void*>(&k_classic<T, V, true, EX>), ring_slot_classic(V, (int)sizeof(T)),
                       p.opts, &rg, &dyn, &ring);
    if (rc != LAP5CG_OK) return rc;
    const void* fn = reinterpret_cast<const void*>(&k_classic<T, V, true, EX>);
    if constexpr (RingOnly<T, V>::value) {
      if (!ring) return LAP5CG_ERR_UNSUPPORTED;
    } else if (!ring) {
      fn = reinterpret_cast<const void*>(&k_classic<T, V, false, EX>);
    }
    rc = plan_units(fn, p.nx, p.ny, V, p.opts, dyn, &cfg, row_align);
    if (rc != LAP5CG_OK) return rc;
    if (ring && p.opts.ring_slots == 0 && cfg.seg_rows < kRingMinRows) {  // short units: register march
      if constexpr (RingOnly<T, V>::value) {
        return LAP5CG_ERR_UNSUPPORTED;  // the caller narrows the lane vector
      } else {
        ring = false;
        rg.S = 0;
        dyn = 0;
        fn = reinterpret_cast<const void*>(&k_classic<T, V, false, EX>);
        rc = plan_units(fn, p.nx, p.ny, V, p.opts, dyn, &cfg, row_align);
        if (rc != LAP5CG_OK) return rc;
      }
    }
    ClassicArgs<T> a;
    a.c = make_common(p, cfg, rg);
    a.b = Grid<const T>{static_cast<const T*>(p.b), p.ld};
    a.x = Grid<T>{static_cast<T*>(p.x), p.ld};
    a.r = Grid<T>{vecp(0), p.ldw};
    a.p0 = Grid<T>{vecp(1), p.ldw};
    a.p1 = Grid<T>{vecp(2), p.ldw};
    a.z = Grid<T>{vecp(3), p.ldw};
    int sz = p.opts.store_z;
    if (sz < 0) sz = (sizeof(T) == 8) ? 1 : 0;  // binary64 is FP64-pipe bound: trade bytes for DP ops
    a.store_z = sz;
    void* args[] = {&a};
    return cooperative_launch(fn, cfg, args, st, rg);
  } else if constexpr (RingOnly<T, V>::value) {
    return LAP5CG_ERR_UNSUPPORTED;  // NewCG keeps six vectors live: narrow lane vectors only
  } else {
    RingGeom rg;
    size_t dyn = 0;
    bool ring = false;
    // the stabilised form (host-checked: never with exact dot products)
    const bool stab = p.opts.stabilized != 0 && !EX;
    const void* fn_ring = stab ? reinterpret_cast<const void*>(&k_newcg<T, V, true, EX, !EX>)
                               : reinterpret_cast<const void*>(&k_newcg<T, V, true, EX>);
    const void* fn_march = stab ? reinterpret_cast<const void*>(&k_newcg<T, V, false, EX, !EX>)
                                : reinterpret_cast<const void*>(&k_newcg<T, V, false, EX>);
    int rc = pick_ring(fn_ring, ring_slot_newcg(V, (int)sizeof(T)), p.opts, &rg, &dyn, &ring);
    if (rc != LAP5CG_OK) return rc;
    const void* fn = ring ? fn_ring : fn_march;
    rc = plan_units(fn, p.nx, p.ny, V, p.opts, dyn, &cfg, row_align);
    if (rc != LAP5CG_OK) return rc;
    if (ring && p.opts.ring_slots == 0 && cfg.seg_rows < kRingMinRows) {  // short units: register march
      ring = false;
      rg.S = 0;
      dyn = 0;
      fn = fn_march;
      rc = plan_units(fn, p.nx, p.ny, V, p.opts, dyn, &cfg, row_align);
      if (rc != LAP5CG_OK) return rc;
    }
    NewcgArgs<T> a;
    a.c = make_common(p, cfg, rg);
    a.b = Grid<const T>{static_cast<const T*>(p.b), p.ld};
    a.x = Grid<T>{static_cast<T*>(p.x), p.ld};
    a.r = Grid<T>{vecp(0), p.ldw};
    a.w0 = Grid<T>{vecp(1), p.ldw};
    a.w1 = Grid<T>{vecp(2), p.ldw};
    a.z = Grid<T>{vecp(3), p.ldw};
    a.q = Grid<T>{vecp(4), p.ldw};
    a.p = Grid<T>{vecp(5), p.ldw};
    a.rr_period = p.opts.rr_period;
    void* args[] = {&a};
    return cooperative_launch(fn, cfg, args, st, rg);
  }
}

}  // namespace lap5
