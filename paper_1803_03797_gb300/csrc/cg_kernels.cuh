// cg_kernels.cuh -- persistent, fused CG kernels (Algorithm 1 and Algorithm 2
// of arxiv 1803.03797) for one grid, one launch per solve.
//
// Work decomposition: the grid is cut into strips of 32*V columns; each strip
// into row segments; a (strip, segment) pair is a warp unit.  A warp marches
// its unit row by row keeping three rows of the stencil operand in registers
// (a register line buffer: the GPU counterpart of the paper's line-buffer /
// window-buffer pipeline, Sec. II-B), takes west/east neighbours by warp
// shuffles and the strip's halo columns by two scalar loads.  Units are owned
// by the same warp in every pass, so only halo values cross warps; they are
// published by the grid barrier that separates passes.  Every other pass
// marches rows in the opposite direction so the rows touched last by one pass
// are still in L2 when the next pass starts.
//
// All scalars (alpha, beta, gamma, delta) and the convergence test stay on the
// device: each reduction ends in a grid barrier after which every CTA holds the
// same totals (fixed summation order) and takes the same decision.
#pragma once

#include "common.cuh"
#include "ring.cuh"
#include "repro.cuh"

namespace lap5 {

// Shared solver state passed to every kernel.
struct SolveCommon {
  int nx, ny;
  Units un;
  Ctl* ctl;
  lap5cg_info* info;
  double* history;
  double tol;
  int maxit;
  int true_res;
  long long timeout_ns;
  RingGeom rg;     // shared-memory row ring (rg.S == 0: register march)
  int* err;        // error word: ring wait timeouts are recorded here
  int* abort_flag; // grid teams: set with err so every CTA leaves at its next barrier
};

// The warp's ring in the kernel's dynamic shared memory (S == 0: disabled).
__device__ __forceinline__ void ring_setup(WarpRing& ring, const SolveCommon& c, unsigned char* dsm) {
  if (c.rg.S > 0) {
    ring.init(dsm + (size_t)(threadIdx.x >> 5) * (size_t)c.rg.warp_bytes, c.rg, c.timeout_ns, c.err, c.abort_flag);
  } else {
    ring.S = 0;
  }
}

// Per-thread bookkeeping of a persistent solve: this warp's index among the
// team's warps and the pass counter.
struct Walker {
  int lane, gw, nw;
  int pc;  // pass counter: odd passes march in reverse
  __device__ __forceinline__ void init(int team_rank, int team_size) {
    lane = threadIdx.x & 31;
    const int wpc = blockDim.x >> 5;
    gw = team_rank * wpc + (threadIdx.x >> 5);
    nw = team_size * wpc;
    pc = 0;
  }
  __device__ __forceinline__ bool rev() const { return (pc & 1) != 0; }
};

// Field loader: the stencil operand is a stored vector g.
template <int V, class T, class M>
__device__ __forceinline__ void field_plain(const Grid<T>& g, int nx, int ny, int j, int x, int xs, int lane,
                                            FRow<V, M>& f) {
  if (j < 0 || j >= ny) { f.zero(); return; }
  load_row<V>(g, j, x, nx, f.f);
  f.hl = (lane == 0) ? load_one<T, M>(g, j, xs - 1, nx) : M(0);
  f.hr = (lane == 31) ? load_one<T, M>(g, j, xs + 32 * V, nx) : M(0);
}

// Info writer (team rank 0, thread 0).  status_local is the status all CTAs
// agreed on; an aborted solve reports the error recorded in the control block.
__device__ __forceinline__ void write_info(const SolveCommon& c, int team_rank, int status_local, bool aborted,
                                           int iters, int outer, double gamma, double bb, double relres_true) {
  if (team_rank != 0 || threadIdx.x != 0) return;
  lap5cg_info inf;
  int st = status_local;
  if (aborted) {
    st = atomicAdd(&c.ctl->status, 0);
    if (st == 0) st = LAP5CG_ERR_SYNC_TIMEOUT;
  } else if (c.err) {
    const int e = atomicAdd(c.err, 0);
    if (e != 0) st = e;
  }
  inf.status = st;
  inf.iters = iters;
  inf.outer_iters = outer;
  inf.pad = 0;
  inf.relres_recursive = (bb > 0.0) ? sqrt(gamma / bb) : 0.0;
  inf.relres_true = relres_true;
  *c.info = inf;
}

// ---------------------------------------------------------------------------
// Common passes.
// ---------------------------------------------------------------------------

// r = b - A x (x is the stencil operand); accumulates (b,b) and (r,r).
// When r is null only the dot products are formed (true-residual check).
template <int V, class TB, class TX, class TR, class Acc>
__device__ __forceinline__ void pass_residual(const SolveCommon& c, Walker& wk, const Grid<const TB>& b,
                                              const Grid<TX>& x, const Grid<TR>& r, Acc& abb, Acc& arr) {
  using M = typename Math<TX>::type;
  struct D { M b[V]; };
  for (int u = wk.gw; u < c.un.nunits; u += wk.nw) {
    int s, y0, y1;
    unit_bounds(c.un, u, c.ny, s, y0, y1);
    const int xs = s * 32 * V, xl = Lanes<V>::first(xs, wk.lane);
    const int nval = c.nx - xl;  // columns from xl to the grid edge
    auto field = [&](int j, FRow<V, M>& f) { field_plain<V>(x, c.nx, c.ny, j, xl, xs, wk.lane, f); };
    auto load = [&](int j, D& d) { load_row<V>(b, j, xl, c.nx, d.b); };
    auto finish = [&](int j, const D& d, const FRow<V, M>& S, const FRow<V, M>& C, const FRow<V, M>& N) {
      M ax[V], rv[V];
      stencil_row<V>(S, C, N, wk.lane, ax);
#pragma unroll
      for (int k = 0; k < V; ++k) rv[k] = d.b[k] - ax[k];
      acc_dot<V>(abb, j, d.b, d.b, nval);
      acc_dot<V>(arr, j, rv, rv, nval);
      if (r.ptr) store_row<V>(r, j, xl, c.nx, rv);
    };
    march<V, M, D>(y0, y1, wk.rev(), field, load, finish);
  }
  ++wk.pc;
}

// x = 0 over the interior (b = 0 case).
template <int V, class TX>
__device__ __forceinline__ void pass_zero(const SolveCommon& c, const Units& un, Walker& wk, const Grid<TX>& x) {
  using M = typename Math<TX>::type;
  for (int u = wk.gw; u < un.nunits; u += wk.nw) {
    int s, y0, y1;
    unit_bounds(un, u, c.ny, s, y0, y1);
    const int xl = Lanes<V>::first(s * 32 * V, wk.lane);
    M zv[V];
#pragma unroll
    for (int k = 0; k < V; ++k) zv[k] = M(0);
    for (int j = y0; j < y1; ++j) store_row<V>(x, j, xl, c.nx, zv);
  }
  ++wk.pc;
}

// ---------------------------------------------------------------------------
// Algorithm 1, fused into two passes per iteration.
//   phase P: p = r + beta p_old on the unit plus halo (beta = 0 and p_old
//            unread in the first iteration), store p, y = A p, store z = y
//            (store_z) and accumulate (p, A p);         -> alpha
//   phase R: x += alpha p; r -= alpha z (z read, or A p recomputed from p with
//            its halo); accumulate (r, r)               -> beta, convergence
// p is double-buffered: phase P reads the old p at halo points that a
// neighbouring warp rewrites in the same pass.
// ---------------------------------------------------------------------------
template <class T>
struct ClassicArgs {
  SolveCommon c;
  Grid<const T> b;
  Grid<T> x, r, p0, p1, z;
  int store_z;
};

template <class T, int V, bool R, bool EX = false, class Team>
__device__ void classic_solve(const ClassicArgs<T>& a, Team& tm, double* red, unsigned char* dsm) {
  using M = typename Math<T>::type;
  // EX: reproducible (exact) dot products
  using Acc = typename std::conditional<EX, AccExact, typename AccOf<M>::type>::type;
  const SolveCommon& c = a.c;
  Walker wk;
  wk.init(tm.rank(), tm.size());
  WarpRing ring;
  ring_setup(ring, c, dsm);

  int status = LAP5CG_NOT_CONVERGED, iters = 0;
  double bb = 0.0, gamma = 0.0, relres_true = nan("");
  bool aborted = false;
  bool pending = false;   // a deferred x update is outstanding
  double alpha_prev = 0.0;
  Grid<T> plast = a.p0;

  {  // r = b - A x0, (b, b), (r, r)
    Acc abb = make_acc<Acc>(tm, 0, c.ny, wk.rev()), arr = make_acc<Acc>(tm, 1, c.ny, wk.rev());
    pass_residual<V>(c, wk, a.b, a.x, a.r, abb, arr);
    double o[2];
    if (!acc_reduce<2>(tm, {&abb, &arr}, o, red)) { aborted = true; goto done; }
    bb = o[0];
    gamma = o[1];
  }
  if (!isfinite(bb)) { status = LAP5CG_ERR_NONFINITE; relres_true = nan(""); goto done; }
  if (bb == 0.0) {
    pass_zero<V>(c, c.un, wk, a.x);
    status = LAP5CG_OK;
    gamma = 0.0;
    relres_true = 0.0;
    goto done;
  }
  {
    const double thr = c.tol > 0.0 ? c.tol * c.tol * bb : 0.0;
    if (c.history && tm.rank() == 0 && threadIdx.x == 0) c.history[0] = sqrt(gamma / bb);
    if (!isfinite(gamma)) { status = LAP5CG_ERR_NONFINITE; goto truecheck; }
    if (gamma <= thr) { status = LAP5CG_OK; goto truecheck; }
    double beta = 0.0;
    int cur = 0;  // p_old lives in p[cur], the new p goes to p[cur ^ 1]
    // With z stored, x += alpha p of iteration k is applied in phase P of
    // iteration k+1, which reads p_k anyway; phase R then streams only r and z.
    // The last update is applied after the loop.  Same operands, same result.
    const bool defer = a.store_z != 0;
    while (iters < c.maxit) {
      const bool first = (iters == 0);
      const Grid<T> pold = cur ? a.p1 : a.p0;
      const Grid<T> pnew = cur ? a.p0 : a.p1;
      const bool upd_x = defer && !first;  // apply iteration k-1's x update in this phase P
      const M ap_prev = (M)alpha_prev;
      // ---------------- phase P ----------------
      double pap;
      {
        Acc acc = make_acc<Acc>(tm, 0, c.ny, wk.rev());
        const M bm = (M)beta;
        struct D { int dummy; };
        if constexpr (R) {
          const RingVec vv[3] = {
              {reinterpret_cast<const unsigned char*>(a.r.ptr), a.r.ld, (int)sizeof(T), RV_HALO | RV_ALWAYS},
              {first ? nullptr : reinterpret_cast<const unsigned char*>(pold.ptr), pold.ld, (int)sizeof(T),
               RV_HALO | RV_ALWAYS},
              {upd_x ? reinterpret_cast<const unsigned char*>(a.x.ptr) : nullptr, a.x.ld, (int)sizeof(T), 0}};
          int off[3];
          ring_layout<V>(vv, off);
          ring.fence_global_to_async();
          for (int u = wk.gw; u < c.un.nunits; u += wk.nw) {
            int s, y0, y1;
            unit_bounds(c.un, u, c.ny, s, y0, y1);
            const int xs = s * 32 * V, xl = Lanes<V>::first(xs, wk.lane);
            const int nval = c.nx - xl;  // columns from xl to the grid edge
            auto field = [&](int j, const unsigned char* sl, FRow<V, M>& f) {
              M rv[V];
              ring_lane<V, T>(sl, off[0], true, wk.lane, xl, c.nx, rv);
              const M hr = ring_halo<V, T, M>(sl, off[0], wk.lane, xs, c.nx);
              if (first) {
#pragma unroll
                for (int k = 0; k < V; ++k) f.f[k] = rv[k];
                f.hl = hr;
              } else {
                M pv[V];
                ring_lane<V, T>(sl, off[1], true, wk.lane, xl, c.nx, pv);
                const M hp = ring_halo<V, T, M>(sl, off[1], wk.lane, xs, c.nx);
#pragma unroll
                for (int k = 0; k < V; ++k) f.f[k] = fmx(bm, pv[k], rv[k]);
                f.hl = fmx(bm, hp, hr);  // one operation serves both halo lanes
                if (upd_x && j >= y0 && j < y1) {  // deferred x += alpha_prev p_prev on the unit's rows
                  M xv[V];
                  ring_lane<V, T>(sl, off[2], false, wk.lane, xl, c.nx, xv);
#pragma unroll
                  for (int k = 0; k < V; ++k) xv[k] = fmx(ap_prev, pv[k], xv[k]);
                  store_row<V>(a.x, j, xl, c.nx, xv);
                }
              }
              f.hr = f.hl;
            };
            auto finish = [&](int j, const unsigned char*, const FRow<V, M>& S, const FRow<V, M>& C,
                              const FRow<V, M>& N) {
              M ap[V];
              stencil_row<V>(S, C, N, wk.lane, ap);
              store_row<V>(pnew, j, xl, c.nx, C.f);
              if (a.store_z) store_row<V>(a.z, j, xl, c.nx, ap);
              acc_dot<V>(acc, j, C.f, ap, nval);
            };
            march_ring<V, M>(ring, c.ny, xs, y0, y1, wk.rev(), vv, off, field, finish);
          }
        } else
        for (int u = wk.gw; u < c.un.nunits; u += wk.nw) {
          int s, y0, y1;
          unit_bounds(c.un, u, c.ny, s, y0, y1);
          const int xs = s * 32 * V, xl = Lanes<V>::first(xs, wk.lane);
          const int nval = c.nx - xl;  // columns from xl to the grid edge
          auto field = [&](int j, FRow<V, M>& f) {
            if (j < 0 || j >= c.ny) { f.zero(); return; }
            M rv[V];
            load_row<V>(a.r, j, xl, c.nx, rv);
            M hlr = (wk.lane == 0) ? load_one<T, M>(a.r, j, xs - 1, c.nx) : M(0);
            M hrr = (wk.lane == 31) ? load_one<T, M>(a.r, j, xs + 32 * V, c.nx) : M(0);
            if (first) {
#pragma unroll
              for (int k = 0; k < V; ++k) f.f[k] = rv[k];
              f.hl = hlr;
              f.hr = hrr;
            } else {
              M pv[V];
              load_row<V>(pold, j, xl, c.nx, pv);
              const M hlp = (wk.lane == 0) ? load_one<T, M>(pold, j, xs - 1, c.nx) : M(0);
              const M hrp = (wk.lane == 31) ? load_one<T, M>(pold, j, xs + 32 * V, c.nx) : M(0);
#pragma unroll
              for (int k = 0; k < V; ++k) f.f[k] = fmx(bm, pv[k], rv[k]);
              f.hl = fmx(bm, hlp, hlr);
              f.hr = fmx(bm, hrp, hrr);
              if (upd_x && j >= y0 && j < y1) {  // deferred x += alpha_prev p_prev on the unit's rows
                M xv[V];
                load_row<V>(a.x, j, xl, c.nx, xv);
#pragma unroll
                for (int k = 0; k < V; ++k) xv[k] = fmx(ap_prev, pv[k], xv[k]);
                store_row<V>(a.x, j, xl, c.nx, xv);
              }
            }
          };
          auto load = [&](int, D&) {};
          auto finish = [&](int j, const D&, const FRow<V, M>& S, const FRow<V, M>& C, const FRow<V, M>& N) {
            M ap[V];
            stencil_row<V>(S, C, N, wk.lane, ap);
            store_row<V>(pnew, j, xl, c.nx, C.f);
            if (a.store_z) store_row<V>(a.z, j, xl, c.nx, ap);
            acc_dot<V>(acc, j, C.f, ap, nval);
          };
          march<V, M, D>(y0, y1, wk.rev(), field, load, finish);
        }
        ++wk.pc;
        double o[1];
        if (!acc_reduce<1>(tm, {&acc}, o, red)) { aborted = true; goto done; }
        pap = o[0];
      }
      if (!(pap > 0.0) || !isfinite(pap)) { status = LAP5CG_ERR_BREAKDOWN; goto truecheck; }
      {
        const double alpha = gamma / pap;
        const M am = (M)alpha;
        Acc acc = make_acc<Acc>(tm, 0, c.ny, wk.rev());
        if constexpr (R) {
          ring.fence_global_to_async();
          if (a.store_z) {
            const RingVec vv[2] = {{reinterpret_cast<const unsigned char*>(a.r.ptr), a.r.ld, (int)sizeof(T), 0},
                                   {reinterpret_cast<const unsigned char*>(a.z.ptr), a.z.ld, (int)sizeof(T), 0}};
            int off[2];
            ring_layout<V>(vv, off);
            for (int u = wk.gw; u < c.un.nunits; u += wk.nw) {
              int s, y0, y1;
              unit_bounds(c.un, u, c.ny, s, y0, y1);
              const int xs = s * 32 * V, xl = Lanes<V>::first(xs, wk.lane);
              const int nval = c.nx - xl;  // columns from xl to the grid edge
              auto finish = [&](int j, const unsigned char* sl) {
                M rv[V], zv[V];
                ring_lane<V, T>(sl, off[0], false, wk.lane, xl, c.nx, rv);
                ring_lane<V, T>(sl, off[1], false, wk.lane, xl, c.nx, zv);
#pragma unroll
                for (int k = 0; k < V; ++k) rv[k] = fmx(-am, zv[k], rv[k]);
                acc_dot<V>(acc, j, rv, rv, nval);
                store_row<V>(a.r, j, xl, c.nx, rv);
              };
              stream_ring<V>(ring, c.ny, xs, y0, y1, wk.rev(), vv, off, finish);
            }
          } else {
            const RingVec vv[3] = {
                {reinterpret_cast<const unsigned char*>(pnew.ptr), pnew.ld, (int)sizeof(T), RV_HALO | RV_ALWAYS},
                {reinterpret_cast<const unsigned char*>(a.x.ptr), a.x.ld, (int)sizeof(T), 0},
                {reinterpret_cast<const unsigned char*>(a.r.ptr), a.r.ld, (int)sizeof(T), 0}};
            int off[3];
            ring_layout<V>(vv, off);
            for (int u = wk.gw; u < c.un.nunits; u += wk.nw) {
              int s, y0, y1;
              unit_bounds(c.un, u, c.ny, s, y0, y1);
              const int xs = s * 32 * V, xl = Lanes<V>::first(xs, wk.lane);
              const int nval = c.nx - xl;  // columns from xl to the grid edge
              auto field = [&](int, const unsigned char* sl, FRow<V, M>& f) {
                ring_lane<V, T>(sl, off[0], true, wk.lane, xl, c.nx, f.f);
                f.hl = ring_halo<V, T, M>(sl, off[0], wk.lane, xs, c.nx);
                f.hr = f.hl;
              };
              auto finish = [&](int j, const unsigned char* sl, const FRow<V, M>& S, const FRow<V, M>& C,
                                const FRow<V, M>& N) {
                M ap[V], xv[V], rv[V];
                stencil_row<V>(S, C, N, wk.lane, ap);
                ring_lane<V, T>(sl, off[1], false, wk.lane, xl, c.nx, xv);
                ring_lane<V, T>(sl, off[2], false, wk.lane, xl, c.nx, rv);
#pragma unroll
                for (int k = 0; k < V; ++k) {
                  xv[k] = fmx(am, C.f[k], xv[k]);
                  rv[k] = fmx(-am, ap[k], rv[k]);
                }
                acc_dot<V>(acc, j, rv, rv, nval);
                store_row<V>(a.x, j, xl, c.nx, xv);
                store_row<V>(a.r, j, xl, c.nx, rv);
              };
              march_ring<V, M>(ring, c.ny, xs, y0, y1, wk.rev(), vv, off, field, finish);
            }
          }
        } else
        for (int u = wk.gw; u < c.un.nunits; u += wk.nw) {
          int s, y0, y1;
          unit_bounds(c.un, u, c.ny, s, y0, y1);
          const int xs = s * 32 * V, xl = Lanes<V>::first(xs, wk.lane);
          const int nval = c.nx - xl;  // columns from xl to the grid edge
          if (a.store_z) {
            struct D { M r[V], z[V]; };
            auto load = [&](int j, D& d) {
              load_row<V>(a.r, j, xl, c.nx, d.r);
              load_row<V>(a.z, j, xl, c.nx, d.z);
            };
            auto finish = [&](int j, const D& d) {
              M rv[V];
#pragma unroll
              for (int k = 0; k < V; ++k) rv[k] = fmx(-am, d.z[k], d.r[k]);
              acc_dot<V>(acc, j, rv, rv, nval);
              store_row<V>(a.r, j, xl, c.nx, rv);
            };
            stream_rows<D>(y0, y1, wk.rev(), load, finish);
          } else {
            struct D { M x[V], r[V]; };
            auto field = [&](int j, FRow<V, M>& f) { field_plain<V>(pnew, c.nx, c.ny, j, xl, xs, wk.lane, f); };
            auto load = [&](int j, D& d) {
              load_row<V>(a.x, j, xl, c.nx, d.x);
              load_row<V>(a.r, j, xl, c.nx, d.r);
            };
            auto finish = [&](int j, const D& d, const FRow<V, M>& S, const FRow<V, M>& C, const FRow<V, M>& N) {
              M ap[V], xv[V], rv[V];
              stencil_row<V>(S, C, N, wk.lane, ap);
#pragma unroll
              for (int k = 0; k < V; ++k) {
                xv[k] = fmx(am, C.f[k], d.x[k]);
                rv[k] = fmx(-am, ap[k], d.r[k]);
              }
              acc_dot<V>(acc, j, rv, rv, nval);
              store_row<V>(a.x, j, xl, c.nx, xv);
              store_row<V>(a.r, j, xl, c.nx, rv);
            };
            march<V, M, D>(y0, y1, wk.rev(), field, load, finish);
          }
        }
        ++wk.pc;
        double o[1];
        if (!acc_reduce<1>(tm, {&acc}, o, red)) { aborted = true; goto done; }
        const double gnew = o[0];
        ++iters;
        if (defer) {
          pending = true;
          alpha_prev = alpha;
          plast = pnew;
        }
        if (c.history && tm.rank() == 0 && threadIdx.x == 0) c.history[iters] = sqrt(gnew / bb);
        if (!isfinite(gnew)) { status = LAP5CG_ERR_NONFINITE; gamma = gnew; goto finalx; }
        beta = gnew / gamma;
        gamma = gnew;
        cur ^= 1;
        if (gnew <= thr) { status = LAP5CG_OK; goto finalx; }
      }
    }
  }
finalx:
  if (pending) {  // the deferred x += alpha p of the last iteration
    const M am = (M)alpha_prev;
    for (int u = wk.gw; u < c.un.nunits; u += wk.nw) {
      int s, y0, y1;
      unit_bounds(c.un, u, c.ny, s, y0, y1);
      const int xl = Lanes<V>::first(s * 32 * V, wk.lane);
      struct D { M x[V], p[V]; };
      auto load = [&](int j, D& d) {
        load_row<V>(a.x, j, xl, c.nx, d.x);
        load_row<V>(plast, j, xl, c.nx, d.p);
      };
      auto finish = [&](int j, const D& d) {
        M xv[V];
#pragma unroll
        for (int k = 0; k < V; ++k) xv[k] = fmx(am, d.p[k], d.x[k]);
        store_row<V>(a.x, j, xl, c.nx, xv);
      };
      stream_rows<D>(y0, y1, wk.rev(), load, finish);
    }
    ++wk.pc;
    pending = false;
    if (!tm.sync(red)) { aborted = true; goto done; }
  }
truecheck:
  if (c.true_res) {
    Acc abb = make_acc<Acc>(tm, -1, c.ny, wk.rev()), arr = make_acc<Acc>(tm, 0, c.ny, wk.rev());
    const Grid<T> none{nullptr, 0};
    pass_residual<V>(c, wk, a.b, a.x, none, abb, arr);
    double o[1];
    if (!acc_reduce<1>(tm, {&arr}, o, red)) { aborted = true; goto done; }
    relres_true = sqrt(o[0] / bb);
  }
done:
  if (ring.S > 0) ring.teardown();
  write_info(c, tm.rank(), status, aborted, iters, 0, gamma, bb, relres_true);
}

// ---------------------------------------------------------------------------
// Algorithm 2 (NewCG), one fused pass and one grid reduction per iteration.
//   prologue: r = b - A x0                       (pass 1, (b,b))
//             w = A r, gamma = (r,r), delta = (w,r)   (pass 2)
//   iteration (Algorithm 2's loop body; the prologue's stencil and updates are
//   the first iteration with beta = 0 and z, q, p unread):
//             n = A w from the w tile plus halo, then
//             z = n + beta z, q = w + beta q, p = r + beta p,
//             x += alpha p, r -= alpha q, w_new = w - alpha z,
//             and (r,r), (w_new,r) of the new vectors for the next iteration.
// w is double-buffered because its halo is read while it is rewritten.
// Residual replacement (rr_period > 0) recomputes r = b - A x, w = A r,
// q = A p, z = A q from x and p every rr_period updates.
// ST (the stabilised form): the same pass also accumulates (r_new, q) and
// (p, q) of the p, q it used, and alpha is gamma / (p, A p) with (p, A p) = delta +
// 2 beta (r, q_old) + beta^2 (p_old, q_old) -- equal to Algorithm 2's
// 1/(delta/gamma - beta/alpha_old) in exact arithmetic, without its
// assumption that consecutive residuals are orthogonal (which fails near the
// attainable accuracy).  Still one reduction (of four values) per iteration.
// ---------------------------------------------------------------------------
template <class T>
struct NewcgArgs {
  SolveCommon c;
  Grid<const T> b;
  Grid<T> x, r, w0, w1, z, q, p;
  int rr_period;
};

// q = A p with (r, q) and (p, q) (residual replacement of the stabilised form).
template <int V, class T, class Acc>
__device__ __forceinline__ void pass_q_from_p(const SolveCommon& c, Walker& wk, const Grid<T>& p, const Grid<T>& q,
                                              const Grid<T>& r, Acc& ae, Acc& amu) {
  using M = typename Math<T>::type;
  struct D { M r[V]; };
  for (int u = wk.gw; u < c.un.nunits; u += wk.nw) {
    int s, y0, y1;
    unit_bounds(c.un, u, c.ny, s, y0, y1);
    const int xs = s * 32 * V, xl = Lanes<V>::first(xs, wk.lane);
    const int nval = c.nx - xl;
    auto field = [&](int j, FRow<V, M>& f) { field_plain<V>(p, c.nx, c.ny, j, xl, xs, wk.lane, f); };
    auto load = [&](int j, D& d) { load_row<V>(r, j, xl, c.nx, d.r); };
    auto finish = [&](int j, const D& d, const FRow<V, M>& S, const FRow<V, M>& C, const FRow<V, M>& N) {
      M qv[V];
      stencil_row<V>(S, C, N, wk.lane, qv);
      store_row<V>(q, j, xl, c.nx, qv);
      acc_dot<V>(ae, j, d.r, qv, nval);
      acc_dot<V>(amu, j, C.f, qv, nval);
    };
    march<V, M, D>(y0, y1, wk.rev(), field, load, finish);
  }
  ++wk.pc;
}

// y = A g for a stored g (whole grid), with optional (y, other) / (g, g) sums.
template <int V, class T>
__device__ __forceinline__ void pass_apply(const SolveCommon& c, Walker& wk, const Grid<T>& g, const Grid<T>& y) {
  using M = typename Math<T>::type;
  struct D { int dummy; };
  for (int u = wk.gw; u < c.un.nunits; u += wk.nw) {
    int s, y0, y1;
    unit_bounds(c.un, u, c.ny, s, y0, y1);
    const int xs = s * 32 * V, xl = Lanes<V>::first(xs, wk.lane);
    auto field = [&](int j, FRow<V, M>& f) { field_plain<V>(g, c.nx, c.ny, j, xl, xs, wk.lane, f); };
    auto load = [&](int, D&) {};
    auto finish = [&](int j, const D&, const FRow<V, M>& S, const FRow<V, M>& C, const FRow<V, M>& N) {
      M yv[V];
      stencil_row<V>(S, C, N, wk.lane, yv);
      store_row<V>(y, j, xl, c.nx, yv);
    };
    march<V, M, D>(y0, y1, wk.rev(), field, load, finish);
  }
  ++wk.pc;
}

// w = A r with gamma = (r, r), delta = (w, r).
template <int V, class T, class Acc>
__device__ __forceinline__ void pass_w_from_r(const SolveCommon& c, Walker& wk, const Grid<T>& r, const Grid<T>& w,
                                              Acc& ag, Acc& ad) {
  using M = typename Math<T>::type;
  struct D { int dummy; };
  for (int u = wk.gw; u < c.un.nunits; u += wk.nw) {
    int s, y0, y1;
    unit_bounds(c.un, u, c.ny, s, y0, y1);
    const int xs = s * 32 * V, xl = Lanes<V>::first(xs, wk.lane);
    const int nval = c.nx - xl;  // columns from xl to the grid edge
    auto field = [&](int j, FRow<V, M>& f) { field_plain<V>(r, c.nx, c.ny, j, xl, xs, wk.lane, f); };
    auto load = [&](int, D&) {};
    auto finish = [&](int j, const D&, const FRow<V, M>& S, const FRow<V, M>& C, const FRow<V, M>& N) {
      M wv[V];
      stencil_row<V>(S, C, N, wk.lane, wv);
      store_row<V>(w, j, xl, c.nx, wv);
      acc_dot<V>(ag, j, C.f, C.f, nval);
      acc_dot<V>(ad, j, wv, C.f, nval);
    };
    march<V, M, D>(y0, y1, wk.rev(), field, load, finish);
  }
  ++wk.pc;
}

template <class T, int V, bool R, bool EX = false, bool ST = false, class Team>
__device__ void newcg_solve(const NewcgArgs<T>& a, Team& tm, double* red, unsigned char* dsm) {
  static_assert(!(EX && ST), "the stabilised alpha takes plain dot products");
  using M = typename Math<T>::type;
  // EX: reproducible (exact) dot products
  using Acc = typename std::conditional<EX, AccExact, typename AccOf<M>::type>::type;
  const SolveCommon& c = a.c;
  Walker wk;
  wk.init(tm.rank(), tm.size());
  WarpRing ring;
  ring_setup(ring, c, dsm);

  int status = LAP5CG_NOT_CONVERGED, iters = 0;
  double bb = 0.0, gamma = 0.0, delta = 0.0, alpha = 0.0, beta = 0.0, relres_true = nan("");
  double eps = 0.0, mu = 0.0;  // stabilised form: (r, q_old), (p_old, q_old)
  bool aborted = false;
  int cur = 0;  // current w lives in w[cur]

  {  // r = b - A x
    Acc abb = make_acc<Acc>(tm, 0, c.ny, wk.rev()), arr = make_acc<Acc>(tm, -1, c.ny, wk.rev());
    pass_residual<V>(c, wk, a.b, a.x, a.r, abb, arr);
    double o[1];
    if (!acc_reduce<1>(tm, {&abb}, o, red)) { aborted = true; goto done; }
    bb = o[0];
  }
  if (!isfinite(bb)) { status = LAP5CG_ERR_NONFINITE; goto done; }
  if (bb == 0.0) {
    pass_zero<V>(c, c.un, wk, a.x);
    status = LAP5CG_OK;
    relres_true = 0.0;
    goto done;
  }
  {
    const double thr = c.tol > 0.0 ? c.tol * c.tol * bb : 0.0;
    {  // w = A r, gamma = (r, r), delta = (w, r)
      Acc ag = make_acc<Acc>(tm, 0, c.ny, wk.rev()), ad = make_acc<Acc>(tm, 1, c.ny, wk.rev());
      pass_w_from_r<V>(c, wk, a.r, a.w0, ag, ad);
      double o[2];
      if (!acc_reduce<2>(tm, {&ag, &ad}, o, red)) { aborted = true; goto done; }
      gamma = o[0];
      delta = o[1];
    }
    if (c.history && tm.rank() == 0 && threadIdx.x == 0) c.history[0] = sqrt(gamma / bb);
    if (!isfinite(gamma)) { status = LAP5CG_ERR_NONFINITE; goto truecheck; }
    if (gamma <= thr) { status = LAP5CG_OK; goto truecheck; }
    if (c.maxit <= 0) goto truecheck;
    if (!(delta > 0.0) || !isfinite(delta)) { status = LAP5CG_ERR_BREAKDOWN; goto truecheck; }
    alpha = gamma / delta;  // beta = 0
    beta = 0.0;
    for (;;) {
      const bool first = (iters == 0);
      const Grid<T> w = cur ? a.w1 : a.w0;
      const Grid<T> wn = cur ? a.w0 : a.w1;
      const M am = (M)alpha, bm = (M)beta;
      Acc ag = make_acc<Acc>(tm, 0, c.ny, wk.rev()), ad = make_acc<Acc>(tm, 1, c.ny, wk.rev());
      Acc ae{}, amu{};  // (r_new, q), (p, q): the stabilised form only
      struct D { M z[V], q[V], p[V], x[V], r[V]; };
      if constexpr (R) {
        ring.fence_global_to_async();
        const unsigned char* nz = first ? nullptr : reinterpret_cast<const unsigned char*>(a.z.ptr);
        const unsigned char* nq = first ? nullptr : reinterpret_cast<const unsigned char*>(a.q.ptr);
        const unsigned char* np = first ? nullptr : reinterpret_cast<const unsigned char*>(a.p.ptr);
        const RingVec vv[6] = {
            {reinterpret_cast<const unsigned char*>(w.ptr), w.ld, (int)sizeof(T), RV_HALO | RV_ALWAYS},
            {nz, a.z.ld, (int)sizeof(T), 0},
            {nq, a.q.ld, (int)sizeof(T), 0},
            {np, a.p.ld, (int)sizeof(T), 0},
            {reinterpret_cast<const unsigned char*>(a.x.ptr), a.x.ld, (int)sizeof(T), 0},
            {reinterpret_cast<const unsigned char*>(a.r.ptr), a.r.ld, (int)sizeof(T), 0}};
        int off[6];
        ring_layout<V>(vv, off);
        for (int u = wk.gw; u < c.un.nunits; u += wk.nw) {
          int s, y0, y1;
          unit_bounds(c.un, u, c.ny, s, y0, y1);
          const int xs = s * 32 * V, xl = Lanes<V>::first(xs, wk.lane);
          const int nval = c.nx - xl;  // columns from xl to the grid edge
          auto field = [&](int, const unsigned char* sl, FRow<V, M>& f) {
            ring_lane<V, T>(sl, off[0], true, wk.lane, xl, c.nx, f.f);
            f.hl = ring_halo<V, T, M>(sl, off[0], wk.lane, xs, c.nx);
            f.hr = f.hl;
          };
          auto finish = [&](int j, const unsigned char* sl, const FRow<V, M>& S, const FRow<V, M>& C,
                            const FRow<V, M>& N) {
            M nv[V], zv[V], qv[V], pv[V], xv[V], rv[V], wv[V];
            stencil_row<V>(S, C, N, wk.lane, nv);  // n = A w
            ring_lane<V, T>(sl, off[4], false, wk.lane, xl, c.nx, xv);
            ring_lane<V, T>(sl, off[5], false, wk.lane, xl, c.nx, rv);
            if (!first) {
              ring_lane<V, T>(sl, off[1], false, wk.lane, xl, c.nx, zv);
              ring_lane<V, T>(sl, off[2], false, wk.lane, xl, c.nx, qv);
              ring_lane<V, T>(sl, off[3], false, wk.lane, xl, c.nx, pv);
            }
#pragma unroll
            for (int k = 0; k < V; ++k) {
              if (first) {
                zv[k] = nv[k];
                qv[k] = C.f[k];
                pv[k] = rv[k];
              } else {
                zv[k] = fmx(bm, zv[k], nv[k]);
                qv[k] = fmx(bm, qv[k], C.f[k]);
                pv[k] = fmx(bm, pv[k], rv[k]);
              }
              xv[k] = fmx(am, pv[k], xv[k]);
              rv[k] = fmx(-am, qv[k], rv[k]);
              wv[k] = fmx(-am, zv[k], C.f[k]);
            }
            acc_dot<V>(ag, j, rv, rv, nval);
            acc_dot<V>(ad, j, wv, rv, nval);
            if constexpr (ST) {
              acc_dot<V>(ae, j, rv, qv, nval);
              acc_dot<V>(amu, j, pv, qv, nval);
            }
            store_row<V>(a.z, j, xl, c.nx, zv);
            store_row<V>(a.q, j, xl, c.nx, qv);
            store_row<V>(a.p, j, xl, c.nx, pv);
            store_row<V>(a.x, j, xl, c.nx, xv);
            store_row<V>(a.r, j, xl, c.nx, rv);
            store_row<V>(wn, j, xl, c.nx, wv);
          };
          march_ring<V, M>(ring, c.ny, xs, y0, y1, wk.rev(), vv, off, field, finish);
        }
      } else
      for (int u = wk.gw; u < c.un.nunits; u += wk.nw) {
        int s, y0, y1;
        unit_bounds(c.un, u, c.ny, s, y0, y1);
        const int xs = s * 32 * V, xl = Lanes<V>::first(xs, wk.lane);
        const int nval = c.nx - xl;  // columns from xl to the grid edge
        auto field = [&](int j, FRow<V, M>& f) { field_plain<V>(w, c.nx, c.ny, j, xl, xs, wk.lane, f); };
        auto load = [&](int j, D& d) {
          if (!first) {
            load_row<V>(a.z, j, xl, c.nx, d.z);
            load_row<V>(a.q, j, xl, c.nx, d.q);
            load_row<V>(a.p, j, xl, c.nx, d.p);
          }
          load_row<V>(a.x, j, xl, c.nx, d.x);
          load_row<V>(a.r, j, xl, c.nx, d.r);
        };
        auto finish = [&](int j, const D& d, const FRow<V, M>& S, const FRow<V, M>& C, const FRow<V, M>& N) {
          M nv[V], zv[V], qv[V], pv[V], xv[V], rv[V], wv[V];
          stencil_row<V>(S, C, N, wk.lane, nv);  // n = A w
#pragma unroll
          for (int k = 0; k < V; ++k) {
            if (first) {
              zv[k] = nv[k];
              qv[k] = C.f[k];
              pv[k] = d.r[k];
            } else {
              zv[k] = fmx(bm, d.z[k], nv[k]);
              qv[k] = fmx(bm, d.q[k], C.f[k]);
              pv[k] = fmx(bm, d.p[k], d.r[k]);
            }
            xv[k] = fmx(am, pv[k], d.x[k]);
            rv[k] = fmx(-am, qv[k], d.r[k]);
            wv[k] = fmx(-am, zv[k], C.f[k]);
          }
          acc_dot<V>(ag, j, rv, rv, nval);
          acc_dot<V>(ad, j, wv, rv, nval);
          if constexpr (ST) {
            acc_dot<V>(ae, j, rv, qv, nval);
            acc_dot<V>(amu, j, pv, qv, nval);
          }
          store_row<V>(a.z, j, xl, c.nx, zv);
          store_row<V>(a.q, j, xl, c.nx, qv);
          store_row<V>(a.p, j, xl, c.nx, pv);
          store_row<V>(a.x, j, xl, c.nx, xv);
          store_row<V>(a.r, j, xl, c.nx, rv);
          store_row<V>(wn, j, xl, c.nx, wv);
        };
        march<V, M, D>(y0, y1, wk.rev(), field, load, finish);
      }
      ++wk.pc;
      ++iters;
      cur ^= 1;
      double gnew, dnew;
      if (a.rr_period > 0 && iters % a.rr_period == 0) {
        // residual replacement: r = b - A x; w = A r; q = A p; z = A q
        if (!tm.sync(red)) { aborted = true; goto done; }
        acc_discard<Acc>(tm);  // the fused pass's (r, r), (w, r) are replaced below
        Acc abb = make_acc<Acc>(tm, -1, c.ny, wk.rev()), arr = make_acc<Acc>(tm, -1, c.ny, wk.rev());
        pass_residual<V>(c, wk, a.b, a.x, a.r, abb, arr);
        if (!tm.sync(red)) { aborted = true; goto done; }
        const Grid<T> wr = cur ? a.w1 : a.w0;
        Acc ag2 = make_acc<Acc>(tm, 0, c.ny, wk.rev()), ad2 = make_acc<Acc>(tm, 1, c.ny, wk.rev());
        pass_w_from_r<V>(c, wk, a.r, wr, ag2, ad2);
        if constexpr (ST) {  // q = A p with (r, q), (p, q) of the replaced vectors
          Acc ae2{}, amu2{};
          pass_q_from_p<V>(c, wk, a.p, a.q, a.r, ae2, amu2);
          double o[4];
          if (!acc_reduce<4>(tm, {&ag2, &ad2, &ae2, &amu2}, o, red)) { aborted = true; goto done; }
          gnew = o[0];
          dnew = o[1];
          eps = o[2];
          mu = o[3];
        } else {
          pass_apply<V>(c, wk, a.p, a.q);
          double o[2];
          if (!acc_reduce<2>(tm, {&ag2, &ad2}, o, red)) { aborted = true; goto done; }
          gnew = o[0];
          dnew = o[1];
        }
        pass_apply<V>(c, wk, a.q, a.z);
        if (!tm.sync(red)) { aborted = true; goto done; }
      } else {
        if constexpr (ST) {
          double o[4];
          if (!acc_reduce<4>(tm, {&ag, &ad, &ae, &amu}, o, red)) { aborted = true; goto done; }
          gnew = o[0];
          dnew = o[1];
          eps = o[2];
          mu = o[3];
        } else {
          double o[2];
          if (!acc_reduce<2>(tm, {&ag, &ad}, o, red)) { aborted = true; goto done; }
          gnew = o[0];
          dnew = o[1];
        }
      }
      if (c.history && tm.rank() == 0 && threadIdx.x == 0) c.history[iters] = sqrt(gnew / bb);
      const double gold = gamma;
      gamma = gnew;
      delta = dnew;
      if (!isfinite(gamma)) { status = LAP5CG_ERR_NONFINITE; goto truecheck; }
      if (gamma <= thr) { status = LAP5CG_OK; goto truecheck; }
      if (iters >= c.maxit) break;
      beta = gamma / gold;
      if constexpr (ST) {  // (p, A p) of p = r + beta p_old from the current vectors, in a fixed order
        const double pap = __dadd_rn(__dadd_rn(delta, __dmul_rn(__dmul_rn(2.0, beta), eps)),
                                     __dmul_rn(__dmul_rn(beta, beta), mu));
        if (!(pap > 0.0) || !isfinite(pap)) { status = LAP5CG_ERR_BREAKDOWN; goto truecheck; }
        alpha = gamma / pap;
      } else {
        const double denom = delta / gamma - beta / alpha;  // de-garbled alpha update
        if (!(denom > 0.0) || !isfinite(denom)) { status = LAP5CG_ERR_BREAKDOWN; goto truecheck; }
        alpha = 1.0 / denom;
      }
    }
  }
truecheck:
  if (c.true_res) {
    Acc abb = make_acc<Acc>(tm, -1, c.ny, wk.rev()), arr = make_acc<Acc>(tm, 0, c.ny, wk.rev());
    const Grid<T> none{nullptr, 0};
    pass_residual<V>(c, wk, a.b, a.x, none, abb, arr);
    double o[1];
    if (!acc_reduce<1>(tm, {&arr}, o, red)) { aborted = true; goto done; }
    relres_true = sqrt(o[0] / bb);
  }
done:
  if (ring.S > 0) ring.teardown();
  write_info(c, tm.rank(), status, aborted, iters, 0, gamma, bb, relres_true);
}

}  // namespace lap5
