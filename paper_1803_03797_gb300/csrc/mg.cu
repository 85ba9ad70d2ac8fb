// mg.cu -- preconditioned CG (Algorithm 1 with M) for the 5-point Laplacian
// with one geometric multigrid V-cycle as M^-1, in one persistent launch.
//
// The paper's NewCG is the pipelined CG of Ghysels and Vanroose with M = I;
// the cited method takes a general preconditioner.  Here M^-1 is a V(nu, nu)
// cycle from zero:
//   levels      (nx, ny) -> ((nx-1)/2, (ny-1)/2), coarse (I, J) at fine
//               (2I+1, 2J+1); coarsening stops when a side would be 0;
//   operators   the same 5-point mask on every level (Sec. II-B); with the
//               unscaled mask the coarse correction is e = P A_c^-1 P^T r;
//   transfers   P bilinear interpolation, restriction P^T (weights
//               [1 2 1; 2 4 2; 1 2 1] / 4), points outside a grid count 0;
//   smoother    damped Jacobi x <- x + c (b - A x), c = 0.2 (omega = 4/5),
//               nu sweeps before and after the coarse correction, nu_c
//               sweeps on the coarsest grid.
// The outer solve and its vectors are binary64; the V-cycle runs in TM
// (binary32 or binary64).  PCG: z = M^-1 r, gamma = (r, z), p = z + beta p,
// alpha = gamma / (p, A p); it stops when (r, r) <= tol^2 (b, b), as the
// unpreconditioned solves do.
//
// Work distribution: every pass is a grid-stride sweep (rows over warps,
// columns over lanes) followed by a grid barrier.  Levels with at most
// kMgCtaPoints points run on CTA 0 alone between two grid barriers, with CTA
// barriers between their passes: there a grid barrier would cost more than
// the work.
#include "mg_kernels.cuh"

namespace lap5 {

template <class TM>
__device__ __forceinline__ void pcg_solve(const PcgArgs<TM>& a, const MgLevel<TM>* lv, GridTeam& tm, double* red) {
  constexpr int V = 2;  // binary64 passes: two columns a lane
  const SolveCommon& c = a.c;
  const int lane = threadIdx.x & 31;
  const int wpc = blockDim.x >> 5;
  const Sched grid{(int)blockIdx.x * wpc + (int)(threadIdx.x >> 5), (int)gridDim.x * wpc, lane, false};
  const Sched cta{(int)(threadIdx.x >> 5), wpc, lane, false};
  const MgLevel<TM> L0 = lv[0];
  const Grid<TM> g0b{L0.b, L0.ld}, g0u{L0.u, L0.ld};
  const TM cm = (TM)kMgC;
  int status = LAP5CG_NOT_CONVERGED, iters = 0;
  double bb = 0.0, rr = 0.0, gamma = 0.0, relres_true = nan("");
  bool aborted = false;
  Acc64 arz;
  Vcycle<TM> vc{a.nlev, a.lsmall, a.nu, a.nu_c, lv, tm, red, grid, cta,
                Grid<const double>{a.r.ptr, a.r.ld}, &arz, {}, true, false, 0u};
  Walker wk;
  wk.init(tm.rank(), tm.size());
  int cur = 0;  // p lives in p[cur]

  {  // r = b - A x; (b, b), (r, r); level 0: b = r, u = c b
    Acc64 abb, arr;
    struct D { double b[V]; };
    for (int u = wk.gw; u < c.un.nunits; u += wk.nw) {
      int s, y0, y1;
      unit_bounds(c.un, u, c.ny, s, y0, y1);
      const int xs = s * 32 * V, xl = Lanes<V>::first(xs, wk.lane);
      const int nval = c.nx - xl;
      auto field = [&](int j, FRow<V, double>& f) { field_plain<V>(a.x, c.nx, c.ny, j, xl, xs, wk.lane, f); };
      auto load = [&](int j, D& d) { load_row<V>(a.b, j, xl, c.nx, d.b); };
      auto finish = [&](int j, const D& d, const FRow<V, double>& S, const FRow<V, double>& C,
                        const FRow<V, double>& N) {
        double ax[V], rv[V];
        TM rb[V], ru[V];
        stencil_row<V>(S, C, N, wk.lane, ax);
#pragma unroll
        for (int k = 0; k < V; ++k) {
          rv[k] = d.b[k] - ax[k];
          rb[k] = (TM)rv[k];
          ru[k] = cm * rb[k];
        }
        acc_dot<V>(abb, j, d.b, d.b, nval);
        acc_dot<V>(arr, j, rv, rv, nval);
        store_row<V>(a.r, j, xl, c.nx, rv);
        store_row<V>(g0b, j, xl, c.nx, rb);
        store_row<V>(g0u, j, xl, c.nx, ru);
      };
      march<V, double, D>(y0, y1, wk.rev(), field, load, finish);
    }
    ++wk.pc;
    double v[2] = {abb.value(), arr.value()}, o[2];
    if (!tm.template reduce<2>(v, o, red)) { aborted = true; goto done; }
    bb = o[0];
    rr = o[1];
  }
  if (!isfinite(bb)) { status = LAP5CG_ERR_NONFINITE; goto done; }
  if (bb == 0.0) {
    pass_zero<V>(c, c.un, wk, a.x);
    status = LAP5CG_OK;
    rr = 0.0;
    relres_true = 0.0;
    goto done;
  }
  {
    const double thr = c.tol > 0.0 ? c.tol * c.tol * bb : 0.0;
    if (c.history && tm.rank() == 0 && threadIdx.x == 0) c.history[0] = sqrt(rr / bb);
    if (!isfinite(rr)) { status = LAP5CG_ERR_NONFINITE; goto truecheck; }
    if (rr <= thr) { status = LAP5CG_OK; goto truecheck; }
    for (;;) {
      // z = M^-1 r and (r, z)
      arz = Acc64{};
      if (!vc.run()) { aborted = true; goto done; }
      if (!vc.dot_done) {  // no sweep wrote level 0 (a single level, one sweep): z = u = c b
        for (int u = wk.gw; u < c.un.nunits; u += wk.nw) {
          int s, y0, y1;
          unit_bounds(c.un, u, c.ny, s, y0, y1);
          const int xl = Lanes<V>::first(s * 32 * V, wk.lane);
          for (int j = y0; j < y1; ++j) {
            double rv[V], zv[V];
            TM zt[V];
            load_row<V>(a.r, j, xl, c.nx, rv);
            load_row<V>(Grid<const TM>{vc.it(0), L0.ld}, j, xl, c.nx, zt);
#pragma unroll
            for (int k = 0; k < V; ++k) zv[k] = mg_widen(zt[k]);
            acc_dot<V>(arz, j, rv, zv, c.nx - xl);
          }
        }
      }
      double beta;
      {
        double v[1] = {arz.value()}, o[1];
        if (!tm.template reduce<1>(v, o, red)) { aborted = true; goto done; }
        if (!(o[0] > 0.0) || !isfinite(o[0])) { status = LAP5CG_ERR_BREAKDOWN; goto truecheck; }
        beta = (iters == 0) ? 0.0 : o[0] / gamma;
        gamma = o[0];
      }
      // p = z + beta p (halo included), q = A p, (p, q)
      const Grid<double> pold = cur ? a.p1 : a.p0;
      const Grid<double> pnew = cur ? a.p0 : a.p1;
      const Grid<const TM> gz{vc.it(0), L0.ld};
      const bool first = (iters == 0);
      double alpha;
      {
        Acc64 apq;
        struct D { int dummy; };
        for (int u = wk.gw; u < c.un.nunits; u += wk.nw) {
          int s, y0, y1;
          unit_bounds(c.un, u, c.ny, s, y0, y1);
          const int xs = s * 32 * V, xl = Lanes<V>::first(xs, wk.lane);
          const int nval = c.nx - xl;
          auto zone = [&](int j, int x) -> double {
            return (x < 0 || x >= c.nx) ? 0.0 : mg_widen(gz.row(j)[x]);
          };
          auto pone = [&](int j, int x) -> double { return (x < 0 || x >= c.nx) ? 0.0 : pold.row(j)[x]; };
          auto field = [&](int j, FRow<V, double>& f) {
            if (j < 0 || j >= c.ny) { f.zero(); return; }
            TM zt[V];
            load_row<V>(gz, j, xl, c.nx, zt);
            if (first) {
#pragma unroll
              for (int k = 0; k < V; ++k) f.f[k] = mg_widen(zt[k]);
              f.hl = (wk.lane == 0) ? zone(j, xs - 1) : 0.0;
              f.hr = (wk.lane == 31) ? zone(j, xs + 32 * V) : 0.0;
            } else {
              double pv[V];
              load_row<V>(pold, j, xl, c.nx, pv);
#pragma unroll
              for (int k = 0; k < V; ++k) f.f[k] = __fma_rn(beta, pv[k], mg_widen(zt[k]));
              f.hl = (wk.lane == 0) ? __fma_rn(beta, pone(j, xs - 1), zone(j, xs - 1)) : 0.0;
              f.hr = (wk.lane == 31) ? __fma_rn(beta, pone(j, xs + 32 * V), zone(j, xs + 32 * V)) : 0.0;
            }
          };
          auto load = [&](int, D&) {};
          auto finish = [&](int j, const D&, const FRow<V, double>& S, const FRow<V, double>& C,
                            const FRow<V, double>& N) {
            double qv[V];
            stencil_row<V>(S, C, N, wk.lane, qv);
            store_row<V>(pnew, j, xl, c.nx, C.f);
            store_row<V>(a.q, j, xl, c.nx, qv);
            acc_dot<V>(apq, j, C.f, qv, nval);
          };
          march<V, double, D>(y0, y1, wk.rev(), field, load, finish);
        }
        ++wk.pc;
        double v[1] = {apq.value()}, o[1];
        if (!tm.template reduce<1>(v, o, red)) { aborted = true; goto done; }
        if (!(o[0] > 0.0) || !isfinite(o[0])) { status = LAP5CG_ERR_BREAKDOWN; goto truecheck; }
        alpha = gamma / o[0];
      }
      cur ^= 1;
      // x += alpha p, r -= alpha q, (r, r); level 0: b = r, u = c b
      {
        Acc64 arr;
        struct D { double x[V], r[V], p[V], q[V]; };
        for (int u = wk.gw; u < c.un.nunits; u += wk.nw) {
          int s, y0, y1;
          unit_bounds(c.un, u, c.ny, s, y0, y1);
          const int xl = Lanes<V>::first(s * 32 * V, wk.lane);
          const int nval = c.nx - xl;
          auto load = [&](int j, D& d) {
            load_row<V>(a.x, j, xl, c.nx, d.x);
            load_row<V>(a.r, j, xl, c.nx, d.r);
            load_row<V>(pnew, j, xl, c.nx, d.p);
            load_row<V>(a.q, j, xl, c.nx, d.q);
          };
          auto finish = [&](int j, const D& d) {
            double xv[V], rv[V];
            TM rb[V], ru[V];
#pragma unroll
            for (int k = 0; k < V; ++k) {
              xv[k] = __fma_rn(alpha, d.p[k], d.x[k]);
              rv[k] = __fma_rn(-alpha, d.q[k], d.r[k]);
              rb[k] = (TM)rv[k];
              ru[k] = cm * rb[k];
            }
            acc_dot<V>(arr, j, rv, rv, nval);
            store_row<V>(a.x, j, xl, c.nx, xv);
            store_row<V>(a.r, j, xl, c.nx, rv);
            store_row<V>(g0b, j, xl, c.nx, rb);
            store_row<V>(g0u, j, xl, c.nx, ru);
          };
          stream_rows<D>(y0, y1, wk.rev(), load, finish);
        }
        ++wk.pc;
        double v[1] = {arr.value()}, o[1];
        if (!tm.template reduce<1>(v, o, red)) { aborted = true; goto done; }
        rr = o[0];
        ++iters;
      }
      if (c.history && tm.rank() == 0 && threadIdx.x == 0) c.history[iters] = sqrt(rr / bb);
      if (!isfinite(rr)) { status = LAP5CG_ERR_NONFINITE; goto truecheck; }
      if (rr <= thr) { status = LAP5CG_OK; goto truecheck; }
      if (iters >= c.maxit) break;
    }
  }
truecheck:
  if (c.true_res) {
    Acc64 abb, arr;
    const Grid<double> none{nullptr, 0};
    pass_residual<V>(c, wk, a.b, a.x, none, abb, arr);
    double v[1] = {arr.value()}, o[1];
    if (!tm.template reduce<1>(v, o, red)) { aborted = true; goto done; }
    relres_true = sqrt(o[0] / bb);
  }
done:
  write_info(c, tm.rank(), status, aborted, iters, 0, rr, bb, relres_true);
}

// Pipelined preconditioned CG (Algorithm 2 with M; M = I gives the paper's
// recurrences).  One fused pass and one grid reduction per iteration besides
// the V-cycle: n = A m from the V-cycle's result m = M^-1 w (binary64
// stencil of the converted iterate), then z = n + beta z, q = m + beta q,
// s = w + beta s, p = u + beta p, x += alpha p, r -= alpha s, u -= alpha q,
// w -= alpha z, the dot products (r, u), (w, u), (r, r) of the new vectors,
// and level 0's right-hand side (w) and first sweep for the next V-cycle --
// written into the buffer the pass does not read.
template <class TM>
__device__ __forceinline__ void ppcg_solve(const PcgArgs<TM>& a, const MgLevel<TM>* lv, GridTeam& tm, double* red) {
  constexpr int V = 2;
  const SolveCommon& c = a.c;
  const int lane = threadIdx.x & 31;
  const int wpc = blockDim.x >> 5;
  const Sched grid{(int)blockIdx.x * wpc + (int)(threadIdx.x >> 5), (int)gridDim.x * wpc, lane, false};
  const Sched cta{(int)(threadIdx.x >> 5), wpc, lane, false};
  const MgLevel<TM> L0 = lv[0];
  const Grid<TM> g0b{L0.b, L0.ld};
  const TM cm = (TM)kMgC;
  int status = LAP5CG_NOT_CONVERGED, iters = 0;
  double bb = 0.0, rr = 0.0, gamma = 0.0, delta = 0.0, alpha = 0.0, relres_true = nan("");
  bool aborted = false;
  Vcycle<TM> vc{a.nlev, a.lsmall, a.nu, a.nu_c, lv, tm, red, grid, cta,
                Grid<const double>{a.r.ptr, a.r.ld}, nullptr, {}, true, false, 0u};
  Walker wk;
  wk.init(tm.rank(), tm.size());
  const Grid<double> pp = a.p0;

  {  // r = b - A x; (b, b), (r, r); level 0: b = r, first sweep in u
    Acc64 abb, arr;
    struct D { double b[V]; };
    const Grid<TM> g0u{L0.u, L0.ld};
    for (int u = wk.gw; u < c.un.nunits; u += wk.nw) {
      int s, y0, y1;
      unit_bounds(c.un, u, c.ny, s, y0, y1);
      const int xs = s * 32 * V, xl = Lanes<V>::first(xs, wk.lane);
      const int nval = c.nx - xl;
      auto field = [&](int j, FRow<V, double>& f) { field_plain<V>(a.x, c.nx, c.ny, j, xl, xs, wk.lane, f); };
      auto load = [&](int j, D& d) { load_row<V>(a.b, j, xl, c.nx, d.b); };
      auto finish = [&](int j, const D& d, const FRow<V, double>& S, const FRow<V, double>& C,
                        const FRow<V, double>& N) {
        double ax[V], rv[V];
        TM rb[V], ru[V];
        stencil_row<V>(S, C, N, wk.lane, ax);
#pragma unroll
        for (int k = 0; k < V; ++k) {
          rv[k] = d.b[k] - ax[k];
          rb[k] = (TM)rv[k];
          ru[k] = cm * rb[k];
        }
        acc_dot<V>(abb, j, d.b, d.b, nval);
        acc_dot<V>(arr, j, rv, rv, nval);
        store_row<V>(a.r, j, xl, c.nx, rv);
        store_row<V>(g0b, j, xl, c.nx, rb);
        store_row<V>(g0u, j, xl, c.nx, ru);
      };
      march<V, double, D>(y0, y1, wk.rev(), field, load, finish);
    }
    ++wk.pc;
    double v[2] = {abb.value(), arr.value()}, o[2];
    if (!tm.template reduce<2>(v, o, red)) { aborted = true; goto done; }
    bb = o[0];
    rr = o[1];
  }
  if (!isfinite(bb)) { status = LAP5CG_ERR_NONFINITE; goto done; }
  if (bb == 0.0) {
    pass_zero<V>(c, c.un, wk, a.x);
    status = LAP5CG_OK;
    rr = 0.0;
    relres_true = 0.0;
    goto done;
  }
  {
    const double thr = c.tol > 0.0 ? c.tol * c.tol * bb : 0.0;
    if (c.history && tm.rank() == 0 && threadIdx.x == 0) c.history[0] = sqrt(rr / bb);
    if (!isfinite(rr)) { status = LAP5CG_ERR_NONFINITE; goto truecheck; }
    if (rr <= thr) { status = LAP5CG_OK; goto truecheck; }
    if (c.maxit <= 0) goto truecheck;
    // u = M^-1 r, w = A u; gamma = (r, u), delta = (w, u); level 0: b = w
    if (!vc.run(0)) { aborted = true; goto done; }
    {
      const int s0 = vc.cur[0] ^ 1;  // the next first sweep goes where the iterate is not
      const Grid<const TM> gm{vc.it(0), L0.ld};
      const Grid<TM> g0n{s0 ? L0.v : L0.u, L0.ld};
      Acc64 ag, ad;
      struct D { double r[V]; };
      for (int u = wk.gw; u < c.un.nunits; u += wk.nw) {
        int s, y0, y1;
        unit_bounds(c.un, u, c.ny, s, y0, y1);
        const int xs = s * 32 * V, xl = Lanes<V>::first(xs, wk.lane);
        const int nval = c.nx - xl;
        auto field = [&](int j, FRow<V, double>& f) { field_wide<V>(gm, c.nx, c.ny, j, xl, xs, wk.lane, f); };
        auto load = [&](int j, D& d) { load_row<V>(a.r, j, xl, c.nx, d.r); };
        auto finish = [&](int j, const D& d, const FRow<V, double>& S, const FRow<V, double>& C,
                          const FRow<V, double>& N) {
          double wv[V];
          TM wb[V], wu[V];
          stencil_row<V>(S, C, N, wk.lane, wv);
#pragma unroll
          for (int k = 0; k < V; ++k) {
            wb[k] = (TM)wv[k];
            wu[k] = cm * wb[k];
          }
          acc_dot<V>(ag, j, d.r, C.f, nval);
          acc_dot<V>(ad, j, wv, C.f, nval);
          store_row<V>(a.u, j, xl, c.nx, C.f);
          store_row<V>(a.w, j, xl, c.nx, wv);
          store_row<V>(g0b, j, xl, c.nx, wb);
          store_row<V>(g0n, j, xl, c.nx, wu);
        };
        march<V, double, D>(y0, y1, wk.rev(), field, load, finish);
      }
      ++wk.pc;
      double v[2] = {ag.value(), ad.value()}, o[2];
      if (!tm.template reduce<2>(v, o, red)) { aborted = true; goto done; }
      gamma = o[0];
      delta = o[1];
      vc.cur[0] = s0;
    }
    double beta = 0.0;
    for (;;) {
      // m = M^-1 w
      if (!vc.run(vc.cur[0])) { aborted = true; goto done; }
      const bool first = (iters == 0);
      if (first) {
        if (!(delta > 0.0) || !isfinite(delta) || !(gamma > 0.0)) { status = LAP5CG_ERR_BREAKDOWN; goto truecheck; }
        beta = 0.0;
        alpha = gamma / delta;
      }
      const int s0 = vc.cur[0] ^ 1;  // the next first sweep goes where m is not
      const Grid<const TM> gm{vc.it(0), L0.ld};
      const Grid<TM> g0n{s0 ? L0.v : L0.u, L0.ld};
      double gn, dn;
      {
        Acc64 ag, ad, arr;
        struct D { int dummy; };
        const double am = alpha, bm = beta;
        for (int u = wk.gw; u < c.un.nunits; u += wk.nw) {
          int s, y0, y1;
          unit_bounds(c.un, u, c.ny, s, y0, y1);
          const int xs = s * 32 * V, xl = Lanes<V>::first(xs, wk.lane);
          const int nval = c.nx - xl;
          auto field = [&](int j, FRow<V, double>& f) { field_wide<V>(gm, c.nx, c.ny, j, xl, xs, wk.lane, f); };
          auto load = [&](int, D&) {};
          auto finish = [&](int j, const D&, const FRow<V, double>& S, const FRow<V, double>& C,
                            const FRow<V, double>& N) {
            double nv[V], zv[V], qv[V], sv[V], pv[V], xv[V], rv[V], uv[V], wv[V];
            TM wb[V], wu[V];
            stencil_row<V>(S, C, N, wk.lane, nv);  // n = A m
            load_row<V>(a.x, j, xl, c.nx, xv);
            load_row<V>(a.r, j, xl, c.nx, rv);
            load_row<V>(a.u, j, xl, c.nx, uv);
            load_row<V>(a.w, j, xl, c.nx, wv);
            if (!first) {
              load_row<V>(a.z, j, xl, c.nx, zv);
              load_row<V>(a.q, j, xl, c.nx, qv);
              load_row<V>(a.s, j, xl, c.nx, sv);
              load_row<V>(pp, j, xl, c.nx, pv);
            }
#pragma unroll
            for (int k = 0; k < V; ++k) {
              if (first) {
                zv[k] = nv[k];
                qv[k] = C.f[k];
                sv[k] = wv[k];
                pv[k] = uv[k];
              } else {
                zv[k] = __fma_rn(bm, zv[k], nv[k]);
                qv[k] = __fma_rn(bm, qv[k], C.f[k]);
                sv[k] = __fma_rn(bm, sv[k], wv[k]);
                pv[k] = __fma_rn(bm, pv[k], uv[k]);
              }
              xv[k] = __fma_rn(am, pv[k], xv[k]);
              rv[k] = __fma_rn(-am, sv[k], rv[k]);
              uv[k] = __fma_rn(-am, qv[k], uv[k]);
              wv[k] = __fma_rn(-am, zv[k], wv[k]);
              wb[k] = (TM)wv[k];
              wu[k] = cm * wb[k];
            }
            acc_dot<V>(ag, j, rv, uv, nval);
            acc_dot<V>(ad, j, wv, uv, nval);
            acc_dot<V>(arr, j, rv, rv, nval);
            store_row<V>(a.z, j, xl, c.nx, zv);
            store_row<V>(a.q, j, xl, c.nx, qv);
            store_row<V>(a.s, j, xl, c.nx, sv);
            store_row<V>(pp, j, xl, c.nx, pv);
            store_row<V>(a.x, j, xl, c.nx, xv);
            store_row<V>(a.r, j, xl, c.nx, rv);
            store_row<V>(a.u, j, xl, c.nx, uv);
            store_row<V>(a.w, j, xl, c.nx, wv);
            store_row<V>(g0b, j, xl, c.nx, wb);
            store_row<V>(g0n, j, xl, c.nx, wu);
          };
          march<V, double, D>(y0, y1, wk.rev(), field, load, finish);
        }
        ++wk.pc;
        double v[3] = {ag.value(), ad.value(), arr.value()}, o[3];
        if (!tm.template reduce<3>(v, o, red)) { aborted = true; goto done; }
        gn = o[0];
        dn = o[1];
        rr = o[2];
        ++iters;
        vc.cur[0] = s0;
      }
      if (c.history && tm.rank() == 0 && threadIdx.x == 0) c.history[iters] = sqrt(rr / bb);
      if (!isfinite(rr)) { status = LAP5CG_ERR_NONFINITE; goto truecheck; }
      if (rr <= thr) { status = LAP5CG_OK; goto truecheck; }
      if (iters >= c.maxit) break;
      const double gold = gamma;
      gamma = gn;
      delta = dn;
      beta = gamma / gold;
      const double denom = delta / gamma - beta / alpha;
      if (!(denom > 0.0) || !isfinite(denom) || !(gamma > 0.0)) { status = LAP5CG_ERR_BREAKDOWN; goto truecheck; }
      alpha = 1.0 / denom;
    }
  }
truecheck:
  if (c.true_res) {
    Acc64 abb, arr;
    const Grid<double> none{nullptr, 0};
    pass_residual<V>(c, wk, a.b, a.x, none, abb, arr);
    double v[1] = {arr.value()}, o[1];
    if (!tm.template reduce<1>(v, o, red)) { aborted = true; goto done; }
    relres_true = sqrt(o[0] / bb);
  }
done:
  write_info(c, tm.rank(), status, aborted, iters, 0, rr, bb, relres_true);
}

template <class TM>
__global__ void __launch_bounds__(512) k_pcg(const PcgArgs<TM> a) {
  __shared__ double red[kRedDoubles];
  __shared__ MgLevel<TM> lv[kMgMaxLevels];
  if (threadIdx.x < kMgMaxLevels) lv[threadIdx.x] = a.lv[threadIdx.x];
  __syncthreads();
  GridTeam tm{a.c.ctl, a.c.timeout_ns, 0ull};
  pcg_solve<TM>(a, lv, tm, red);
}

template <class TM>
__global__ void __launch_bounds__(512) k_ppcg(const PcgArgs<TM> a) {
  __shared__ double red[kRedDoubles];
  __shared__ MgLevel<TM> lv[kMgMaxLevels];
  if (threadIdx.x < kMgMaxLevels) lv[threadIdx.x] = a.lv[threadIdx.x];
  __syncthreads();
  GridTeam tm{a.c.ctl, a.c.timeout_ns, 0ull};
  ppcg_solve<TM>(a, lv, tm, red);
}

// Level geometry: sides shrink to (n-1)/2 until one would be 0 (or max levels).
static int mg_levels(int nx, int ny, int max_levels, int* lnx, int* lny) {
  int L = 0;
  while (L < kMgMaxLevels && (max_levels <= 0 || L < max_levels)) {
    lnx[L] = nx;
    lny[L] = ny;
    ++L;
    const int cx = (nx - 1) / 2, cy = (ny - 1) / 2;
    if (cx < 1 || cy < 1) break;
    nx = cx;
    ny = cy;
  }
  return L;
}

static int mg_pitch(int nx) { return (nx + 3) / 4 * 4; }

template <class TM>
static size_t mg_level_bytes(int nx, int ny) {
  int lnx[kMgMaxLevels], lny[kMgMaxLevels];
  const int L = mg_levels(nx, ny, 0, lnx, lny);
  size_t s = 0;
  for (int l = 0; l < L; ++l) s += 3 * align_up((size_t)mg_pitch(lnx[l]) * (size_t)lny[l] * sizeof(TM), kAlign);
  return s;
}

// binary64 vectors: classic r, p0, p1, q; pipelined r, u, w, z, q, s, p
static int mg_vectors(int variant) { return variant == LAP5CG_NEWCG ? 7 : 4; }

size_t ws_bytes_mg(int nx, int ny, int ldw, int variant, int precision) {
  const size_t vec = align_up((size_t)ny * (size_t)ldw * sizeof(double), kAlign);
  const size_t lv = precision == LAP5CG_PREC_MG_F32 ? mg_level_bytes<float>(nx, ny) : mg_level_bytes<double>(nx, ny);
  return kCtlBytes + mg_vectors(variant) * vec + lv;
}

// The classic form as a CUDA graph (mg_graph.cu); *used = false when the
// shape takes the persistent kernel.
template <class TM>
int solve_mg_graph(const SolvePlan& p, const PcgArgs<TM>& a, cudaStream_t st, bool* used);

template <class TM>
static int solve_mg_t(const SolvePlan& p, cudaStream_t st) {
  const size_t vec = align_up((size_t)p.ny * (size_t)p.ldw * sizeof(double), kAlign);
  unsigned char* base = p.ws + kCtlBytes;
  if (cudaMemsetAsync(p.ws, 0, 256, st) != cudaSuccess) return LAP5CG_ERR_CUDA;
  PcgArgs<TM> a;
  int lnx[kMgMaxLevels], lny[kMgMaxLevels];
  a.nlev = mg_levels(p.nx, p.ny, p.opts.mg_levels, lnx, lny);
  unsigned char* lv = base + mg_vectors(p.variant) * vec;
  a.lsmall = a.nlev;
  for (int l = 0; l < a.nlev; ++l) {
    const size_t bytes = align_up((size_t)mg_pitch(lnx[l]) * (size_t)lny[l] * sizeof(TM), kAlign);
    a.lv[l].nx = lnx[l];
    a.lv[l].ny = lny[l];
    a.lv[l].ld = mg_pitch(lnx[l]);
    a.lv[l].b = reinterpret_cast<TM*>(lv);
    a.lv[l].u = reinterpret_cast<TM*>(lv + bytes);
    a.lv[l].v = reinterpret_cast<TM*>(lv + 2 * bytes);
    lv += 3 * bytes;
    if (a.lsmall == a.nlev && (long long)lnx[l] * lny[l] <= kMgCtaPoints) a.lsmall = l;
  }
  a.nu = p.opts.mg_nu > 0 ? p.opts.mg_nu : 2;
  a.nu_c = p.opts.mg_coarse_sweeps > 0 ? p.opts.mg_coarse_sweeps : 8;
  a.b = Grid<const double>{static_cast<const double*>(p.b), p.ld};
  a.x = Grid<double>{static_cast<double*>(p.x), p.ld};
  a.r = Grid<double>{reinterpret_cast<double*>(base), p.ldw};
  a.p0 = Grid<double>{reinterpret_cast<double*>(base + vec), p.ldw};
  a.p1 = Grid<double>{reinterpret_cast<double*>(base + 2 * vec), p.ldw};
  a.q = Grid<double>{reinterpret_cast<double*>(base + 3 * vec), p.ldw};
  if (p.variant == LAP5CG_CLASSIC) {  // one kernel per pass in a device-looped graph
    bool used = false;
    const int grc = solve_mg_graph<TM>(p, a, st, &used);
    if (grc != LAP5CG_OK || used) return grc;
  }
  LaunchCfg cfg;
  const void* fn = p.variant == LAP5CG_NEWCG ? reinterpret_cast<const void*>(&k_ppcg<TM>)
                                             : reinterpret_cast<const void*>(&k_pcg<TM>);
  lap5cg_opts o = p.opts;
  if (o.warps_per_cta <= 0) o.warps_per_cta = 16;  // a wide CTA 0 for the small levels
  int rc = plan_units(fn, p.nx, p.ny, 2, o, 0, &cfg);
  if (rc != LAP5CG_OK) return rc;
  RingGeom rg{0, 0, 0};
  a.c = make_common(p, cfg, rg);
  a.b = Grid<const double>{static_cast<const double*>(p.b), p.ld};
  a.x = Grid<double>{static_cast<double*>(p.x), p.ld};
  a.r = Grid<double>{reinterpret_cast<double*>(base), p.ldw};
  a.p0 = Grid<double>{reinterpret_cast<double*>(base + vec), p.ldw};
  a.p1 = Grid<double>{reinterpret_cast<double*>(base + 2 * vec), p.ldw};
  a.q = Grid<double>{reinterpret_cast<double*>(base + 3 * vec), p.ldw};
  if (p.variant == LAP5CG_NEWCG) {  // r, p (p0), q as above; u, w, z, s after them
    a.u = Grid<double>{reinterpret_cast<double*>(base + 4 * vec), p.ldw};
    a.w = Grid<double>{reinterpret_cast<double*>(base + 5 * vec), p.ldw};
    a.z = Grid<double>{reinterpret_cast<double*>(base + 6 * vec), p.ldw};
    a.s = Grid<double>{reinterpret_cast<double*>(base + 2 * vec), p.ldw};  // p1 is unused: s
  } else {
    a.u = a.w = a.z = a.s = Grid<double>{nullptr, 0};
  }
  void* args[] = {&a};
  return cooperative_launch(fn, cfg, args, st, rg);
}

int solve_mg(const SolvePlan& p, cudaStream_t st) {
  // The pipelined recurrences keep u = M^-1 r only for an exactly linear M: a
  // binary32 V-cycle's rounding breaks the alpha denominator down near a
  // relative residual of 1e-6 (a binary64 restatement with the V-cycle's
  // input and output rounded to binary32 does the same).
  if (p.variant == LAP5CG_NEWCG && p.precision == LAP5CG_PREC_MG_F32) return LAP5CG_ERR_UNSUPPORTED;
  if (p.precision == LAP5CG_PREC_MG_F32) return solve_mg_t<float>(p, st);
  if (p.precision == LAP5CG_PREC_MG_F64) return solve_mg_t<double>(p, st);
  return LAP5CG_ERR_INVALID_ARG;
}

}  // namespace lap5
