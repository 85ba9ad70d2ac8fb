// ir_kernels.cuh -- mixed-precision solve in one persistent launch: an outer
// binary64 iterative-refinement loop around an inner classic CG
// (Algorithm 1 of arxiv 1803.03797) stored in binary32, or with p and r
// stored as bf16.
//
//   outer passes (binary64): x <- x + d with (d, A d), then r = b - A x with
//                          (r, r), (d, r) and, once, (b, b); r is rounded to
//                          the inner storage and becomes the inner right-hand
//                          side.  A step that raised (r, r) is kept only if it
//                          lowered the error's A-norm (see the guard below).
//   inner CG (binary32 arithmetic, Dot2 dot products) on A d = r_in from d = 0,
//   two fused passes per iteration as in the binary64 classic kernel.
// The outer residual, the update of x and their dot products are the only
// binary64 work; the inner iterations move 32 (binary32) or 20 (bf16 p, r)
// bytes per point.
#pragma once

#include "cg_kernels.cuh"

namespace lap5 {

template <class TR>
struct IrArgs {
  SolveCommon c;                 // c.maxit caps the total inner iterations
  Grid<const double> b;
  Grid<double> x;
  Grid<TR> r, p0, p1;            // inner r and p (binary32 or bf16)
  Grid<float> z, d;              // inner A p (stored form) and correction d
  Units uo;                      // warp units of the outer passes (lane vector VO)
  int store_z;
  int max_outer;
  int maxit_inner;
  double tol_inner;
};

// V: lane vector of the inner passes (c.un); VO: lane vector of the binary64
// outer passes (a.uo).  Grid barriers separate every pass, so the two unit
// decompositions never touch the same data concurrently.
template <class TR, int V, int VO, bool R, class Team>
__device__ void ir_solve(const IrArgs<TR>& a, Team& tm, double* red, unsigned char* dsm) {
  using Acc = Acc32;
  const SolveCommon& c = a.c;
  Walker wk;
  wk.init(tm.rank(), tm.size());
  WarpRing ring;
  ring_setup(ring, c, dsm);
  constexpr int ES = (int)sizeof(TR);
  // bf16 p, r: Polak-Ribiere beta (r_new, r_new - r_old) / (r_old, r_old), equal
  // to Algorithm 1's beta in exact arithmetic; it discounts the part of r_new
  // that the bf16 rounding left along r_old
  constexpr bool kPR = (ES == 2);
  // A p stored (zs) only with four columns a lane: the stored form's register
  // march would not fit the register budget with eight
  const int zs = Lanes<V>::G > 1 ? 0 : a.store_z;

  int status = LAP5CG_NOT_CONVERGED, total = 0, outer = 0;
  double bb = 0.0, rr = 0.0, rr_prev = 0.0, relres_true = nan("");
  double dad = 0.0, drn = 0.0;  // (d, A d) and (d, r_new) of the last correction
  bool aborted = false, have_d = false, reverting = false;
  double thr = 0.0;

  for (;;) {
    // ---------------- outer passes (binary64) ----------------
    // x <- x + d is element-wise, but the residual pass reads x at halo
    // points, so the update is a pass of its own followed by a grid barrier:
    // updating x inside the stencil pass would let a neighbour read an
    // already-updated halo value.  (d was published by the barrier that ended
    // the last inner pass.)
    if (have_d && reverting) {  // x - d undoes a rejected correction
      struct DU { double x[VO]; float d[VO]; };
      for (int u = wk.gw; u < a.uo.nunits; u += wk.nw) {
        int s, y0, y1;
        unit_bounds(a.uo, u, c.ny, s, y0, y1);
        const int xl = Lanes<VO>::first(s * 32 * VO, wk.lane);
        auto load = [&](int j, DU& dd) {
          load_row<VO>(a.x, j, xl, c.nx, dd.x);
          load_row<VO>(a.d, j, xl, c.nx, dd.d);
        };
        auto finish = [&](int j, const DU& dd) {
          double xv[VO];
#pragma unroll
          for (int k = 0; k < VO; ++k) xv[k] = dd.x[k] - (double)dd.d[k];
          store_row<VO>(a.x, j, xl, c.nx, xv);
        };
        stream_rows<DU>(y0, y1, wk.rev(), load, finish);
      }
      ++wk.pc;
      if (!tm.sync(red)) { aborted = true; goto done; }
    } else if (have_d) {
      // x += d, and (d, A d) with the binary64 stencil of the binary32 d (a
      // march over d: it reads no x at halo points)
      Acc64 aad;
      struct DU { double x[VO]; };
      for (int u = wk.gw; u < a.uo.nunits; u += wk.nw) {
        int s, y0, y1;
        unit_bounds(a.uo, u, c.ny, s, y0, y1);
        const int xs = s * 32 * VO, xl = Lanes<VO>::first(xs, wk.lane);
        const int nval = c.nx - xl;
        auto field = [&](int j, FRow<VO, double>& f) {
          if (j < 0 || j >= c.ny) { f.zero(); return; }
          float dv[VO];
          load_row<VO>(a.d, j, xl, c.nx, dv);
#pragma unroll
          for (int k = 0; k < VO; ++k) f.f[k] = (double)dv[k];
          const int xh = xs + 32 * VO;
          f.hl = (wk.lane == 0 && xs > 0) ? (double)a.d.row(j)[xs - 1] : 0.0;
          f.hr = (wk.lane == 31 && xh < c.nx) ? (double)a.d.row(j)[xh] : 0.0;
        };
        auto load = [&](int j, DU& dd) { load_row<VO>(a.x, j, xl, c.nx, dd.x); };
        auto finish = [&](int j, const DU& dd, const FRow<VO, double>& S, const FRow<VO, double>& C,
                          const FRow<VO, double>& N) {
          double xv[VO], ad[VO];
          stencil_row<VO>(S, C, N, wk.lane, ad);
#pragma unroll
          for (int k = 0; k < VO; ++k) {
            xv[k] = dd.x[k] + C.f[k];
            if (Lanes<VO>::col(k) < nval) aad.add(C.f[k], ad[k]);
          }
          store_row<VO>(a.x, j, xl, c.nx, xv);
        };
        march<VO, double, DU>(y0, y1, wk.rev(), field, load, finish);
      }
      ++wk.pc;
      double v[1] = {aad.value()}, o[1];
      if (!tm.template reduce<1>(v, o, red)) { aborted = true; goto done; }
      dad = o[0];
    }
    double g_in;
    {
      Acc64 abb, arr, adr;
      Acc32 agi;
      const bool with_d = have_d && !reverting;  // (d, r_new) for the step's energy test
      struct D { double b[VO]; float d[VO]; };
      for (int u = wk.gw; u < a.uo.nunits; u += wk.nw) {
        int s, y0, y1;
        unit_bounds(a.uo, u, c.ny, s, y0, y1);
        const int xs = s * 32 * VO, xl = Lanes<VO>::first(xs, wk.lane);
        const int nval = c.nx - xl;  // columns from xl to the grid edge
        auto field = [&](int j, FRow<VO, double>& f) { field_plain<VO>(a.x, c.nx, c.ny, j, xl, xs, wk.lane, f); };
        auto load = [&](int j, D& dd) {
          load_row<VO>(a.b, j, xl, c.nx, dd.b);
          if (with_d) load_row<VO>(a.d, j, xl, c.nx, dd.d);
        };
        auto finish = [&](int j, const D& dd, const FRow<VO, double>& S, const FRow<VO, double>& C,
                          const FRow<VO, double>& N) {
          double ax[VO];
          float ri[VO];
          stencil_row<VO>(S, C, N, wk.lane, ax);
#pragma unroll
          for (int k = 0; k < VO; ++k) {
            const double rv = dd.b[k] - ax[k];
            ri[k] = quantize<TR>(__double2float_rn(rv));
            if (Lanes<VO>::col(k) < nval) {
              if (outer == 0) abb.add(dd.b[k], dd.b[k]);
              arr.add(rv, rv);
              agi.add(ri[k], ri[k]);
              if (with_d) adr.add((double)dd.d[k], rv);
            }
          }
          store_row<VO>(a.r, j, xl, c.nx, ri);
        };
        march<VO, double, D>(y0, y1, wk.rev(), field, load, finish);
      }
      ++wk.pc;
      double v[4] = {abb.value(), arr.value(), agi.value(), adr.value()}, o[4];
      if (!tm.template reduce<4>(v, o, red)) { aborted = true; goto done; }
      drn = o[3];
      if (outer == 0) {
        bb = o[0];
        if (!isfinite(bb)) { status = LAP5CG_ERR_NONFINITE; goto done; }
        if (bb == 0.0) {
          pass_zero<VO>(c, a.uo, wk, a.x);
          status = LAP5CG_OK;
          rr = 0.0;
          relres_true = 0.0;
          goto done;
        }
        thr = c.tol > 0.0 ? c.tol * c.tol * bb : 0.0;
      }
      rr = o[1];
      g_in = o[2];
      relres_true = sqrt(rr / bb);
      if (c.history && outer <= c.maxit && tm.rank() == 0 && threadIdx.x == 0) c.history[outer] = relres_true;
    }
    if (!isfinite(rr)) { status = LAP5CG_ERR_NONFINITE; goto done; }
    if (reverting) { status = LAP5CG_NOT_CONVERGED; goto done; }
    if (rr <= thr) { status = LAP5CG_OK; goto done; }
    if (outer > 0 && !(rr < rr_prev)) {
      // The FP64 residual did not fall.  Keep the step if it lowered the
      // error's A-norm by at least half of what it claims: the energy falls by
      // (d, r_old) + (d, r_new), with (d, r_old) = (d, r_new) + (d, A d) > 0,
      // so the test is (d, r_new) >= -(d, r_old) / 2.  A truncated CG
      // correction has (d, r_new) = 0 in exact arithmetic; one made of
      // rounding noise has (d, A d) dominant.  Otherwise undo it (x -= d),
      // recompute the residual and stop with the better iterate.
      if (!have_d) { status = LAP5CG_NOT_CONVERGED; goto done; }  // the inner solve made no correction
      const double dro = drn + dad;
      if (!(dro > 0.0 && drn >= -0.5 * dro)) {
        reverting = true;
        have_d = true;
        continue;
      }
    }
    rr_prev = rr;
    if (outer >= a.max_outer || total >= c.maxit) { status = LAP5CG_NOT_CONVERGED; goto done; }

    // ---------------- inner classic CG on A d = r_in, d0 = 0 ----------------
    {
      double gamma = g_in;
      const double thr_in = a.tol_inner * a.tol_inner * gamma;
      double beta = 0.0;
      int cur = 0, k = 0;
      while (k < a.maxit_inner && total < c.maxit && gamma > thr_in) {
        const bool first = (k == 0);
        const Grid<TR> pold = cur ? a.p1 : a.p0;
        const Grid<TR> pnew = cur ? a.p0 : a.p1;
        double pz;
        {  // phase P
          Acc acc;
          const float bm = (float)beta;
          struct D { int dummy; };
          if constexpr (R) {
            const RingVec vv[2] = {
                {reinterpret_cast<const unsigned char*>(a.r.ptr), a.r.ld, ES, RV_HALO | RV_ALWAYS},
                {first ? nullptr : reinterpret_cast<const unsigned char*>(pold.ptr), pold.ld, ES, RV_HALO | RV_ALWAYS}};
            int off[2];
            ring_layout<V>(vv, off);
            ring.fence_global_to_async();
            for (int u = wk.gw; u < c.un.nunits; u += wk.nw) {
              int s, y0, y1;
              unit_bounds(c.un, u, c.ny, s, y0, y1);
              const int xs = s * 32 * V, xl = Lanes<V>::first(xs, wk.lane);
              const int nval = c.nx - xl;  // columns from xl to the grid edge
              auto field = [&](int, const unsigned char* sl, FRow<V, float>& f) {
                float rv[V];
                ring_lane<V, TR>(sl, off[0], true, wk.lane, xl, c.nx, rv);
                const float hr = ring_halo<V, TR, float>(sl, off[0], wk.lane, xs, c.nx);
                if (first) {
#pragma unroll
                  for (int q = 0; q < V; ++q) f.f[q] = rv[q];
                  f.hl = hr;
                } else {
                  float pv[V];
                  ring_lane<V, TR>(sl, off[1], true, wk.lane, xl, c.nx, pv);
                  const float hp = ring_halo<V, TR, float>(sl, off[1], wk.lane, xs, c.nx);
#pragma unroll
                  for (int q = 0; q < V; ++q) f.f[q] = quantize<TR>(fmx(bm, pv[q], rv[q]));
                  f.hl = quantize<TR>(fmx(bm, hp, hr));
                }
                f.hr = f.hl;
              };
              auto finish = [&](int j, const unsigned char*, const FRow<V, float>& S, const FRow<V, float>& C,
                                const FRow<V, float>& N) {
                float ap[V];
                stencil_row<V>(S, C, N, wk.lane, ap);
                store_row<V>(pnew, j, xl, c.nx, C.f);
                if (zs) store_row<V>(a.z, j, xl, c.nx, ap);
                acc_dot<V>(acc, j, C.f, ap, nval);
              };
              march_ring<V, float>(ring, c.ny, xs, y0, y1, wk.rev(), vv, off, field, finish);
            }
          } else
          for (int u = wk.gw; u < c.un.nunits; u += wk.nw) {
            int s, y0, y1;
            unit_bounds(c.un, u, c.ny, s, y0, y1);
            const int xs = s * 32 * V, xl = Lanes<V>::first(xs, wk.lane);
            const int nval = c.nx - xl;  // columns from xl to the grid edge
            auto field = [&](int j, FRow<V, float>& f) {
              if (j < 0 || j >= c.ny) { f.zero(); return; }
              float rv[V];
              load_row<V>(a.r, j, xl, c.nx, rv);
              const float hlr = (wk.lane == 0) ? load_one<TR, float>(a.r, j, xs - 1, c.nx) : 0.f;
              const float hrr = (wk.lane == 31) ? load_one<TR, float>(a.r, j, xs + 32 * V, c.nx) : 0.f;
              if (first) {
#pragma unroll
                for (int q = 0; q < V; ++q) f.f[q] = rv[q];
                f.hl = hlr;
                f.hr = hrr;
              } else {
                float pv[V];
                load_row<V>(pold, j, xl, c.nx, pv);
                const float hlp = (wk.lane == 0) ? load_one<TR, float>(pold, j, xs - 1, c.nx) : 0.f;
                const float hrp = (wk.lane == 31) ? load_one<TR, float>(pold, j, xs + 32 * V, c.nx) : 0.f;
#pragma unroll
                for (int q = 0; q < V; ++q) f.f[q] = quantize<TR>(fmx(bm, pv[q], rv[q]));
                f.hl = quantize<TR>(fmx(bm, hlp, hlr));
                f.hr = quantize<TR>(fmx(bm, hrp, hrr));
              }
            };
            auto load = [&](int, D&) {};
            auto finish = [&](int j, const D&, const FRow<V, float>& S, const FRow<V, float>& C,
                              const FRow<V, float>& N) {
              float ap[V];
              stencil_row<V>(S, C, N, wk.lane, ap);
              store_row<V>(pnew, j, xl, c.nx, C.f);
              if (zs) store_row<V>(a.z, j, xl, c.nx, ap);
              acc_dot<V>(acc, j, C.f, ap, nval);
            };
            march<V, float, D>(y0, y1, wk.rev(), field, load, finish);
          }
          ++wk.pc;
          double v[1] = {acc.value()}, o[1];
          if (!tm.template reduce<1>(v, o, red)) { aborted = true; goto done; }
          pz = o[0];
        }
        if (!(pz > 0.0) || !isfinite(pz)) { status = LAP5CG_ERR_BREAKDOWN; goto done; }
        {  // phase R
          const float am = (float)(gamma / pz);
          Acc acc, aro;  // (r, r) and, for bf16 storage, (r_new, r_old)
          if (R && !zs) {
            const RingVec vv[3] = {
                {reinterpret_cast<const unsigned char*>(pnew.ptr), pnew.ld, ES, RV_HALO | RV_ALWAYS},
                {first ? nullptr : reinterpret_cast<const unsigned char*>(a.d.ptr), a.d.ld, 4, 0},
                {reinterpret_cast<const unsigned char*>(a.r.ptr), a.r.ld, ES, 0}};
            int off[3];
            ring_layout<V>(vv, off);
            ring.fence_global_to_async();
            for (int u = wk.gw; u < c.un.nunits; u += wk.nw) {
              int s, y0, y1;
              unit_bounds(c.un, u, c.ny, s, y0, y1);
              const int xs = s * 32 * V, xl = Lanes<V>::first(xs, wk.lane);
              const int nval = c.nx - xl;  // columns from xl to the grid edge
              auto field = [&](int, const unsigned char* sl, FRow<V, float>& f) {
                ring_lane<V, TR>(sl, off[0], true, wk.lane, xl, c.nx, f.f);
                f.hl = ring_halo<V, TR, float>(sl, off[0], wk.lane, xs, c.nx);
                f.hr = f.hl;
              };
              auto finish = [&](int j, const unsigned char* sl, const FRow<V, float>& S, const FRow<V, float>& C,
                                const FRow<V, float>& N) {
                float ap[V], dv[V], rv[V], ro[V];
                stencil_row<V>(S, C, N, wk.lane, ap);
                ring_lane<V, TR>(sl, off[2], false, wk.lane, xl, c.nx, rv);
                if (!first) ring_lane<V, float>(sl, off[1], false, wk.lane, xl, c.nx, dv);
#pragma unroll
                for (int q = 0; q < V; ++q) {
                  ro[q] = rv[q];
                  dv[q] = first ? __fmul_rn(am, C.f[q]) : fmx(am, C.f[q], dv[q]);
                  rv[q] = quantize<TR>(fmx(-am, ap[q], rv[q]));
                }
                acc_dot<V>(acc, j, rv, rv, nval);
                if constexpr (kPR) acc_dot<V>(aro, j, rv, ro, nval);
                store_row<V>(a.d, j, xl, c.nx, dv);
                store_row<V>(a.r, j, xl, c.nx, rv);
              };
              march_ring<V, float>(ring, c.ny, xs, y0, y1, wk.rev(), vv, off, field, finish);
            }
          } else
          for (int u = wk.gw; u < c.un.nunits; u += wk.nw) {
            int s, y0, y1;
            unit_bounds(c.un, u, c.ny, s, y0, y1);
            const int xs = s * 32 * V, xl = Lanes<V>::first(xs, wk.lane);
            const int nval = c.nx - xl;  // columns from xl to the grid edge
            if (zs) {
              struct D { float p[V], d[V], r[V], z[V]; };
              auto load = [&](int j, D& dd) {
                load_row<V>(pnew, j, xl, c.nx, dd.p);
                if (!first) load_row<V>(a.d, j, xl, c.nx, dd.d);
                load_row<V>(a.r, j, xl, c.nx, dd.r);
                load_row<V>(a.z, j, xl, c.nx, dd.z);
              };
              auto finish = [&](int j, const D& dd) {
                float dv[V], rv[V];
#pragma unroll
                for (int q = 0; q < V; ++q) {
                  dv[q] = first ? __fmul_rn(am, dd.p[q]) : fmx(am, dd.p[q], dd.d[q]);
                  rv[q] = quantize<TR>(fmx(-am, dd.z[q], dd.r[q]));
                }
                acc_dot<V>(acc, j, rv, rv, nval);
                if constexpr (kPR) acc_dot<V>(aro, j, rv, dd.r, nval);
                store_row<V>(a.d, j, xl, c.nx, dv);
                store_row<V>(a.r, j, xl, c.nx, rv);
              };
              stream_rows<D>(y0, y1, wk.rev(), load, finish);
            } else {
              struct D { float d[V], r[V]; };
              auto field = [&](int j, FRow<V, float>& f) { field_plain<V>(pnew, c.nx, c.ny, j, xl, xs, wk.lane, f); };
              auto load = [&](int j, D& dd) {
                if (!first) load_row<V>(a.d, j, xl, c.nx, dd.d);
                load_row<V>(a.r, j, xl, c.nx, dd.r);
              };
              auto finish = [&](int j, const D& dd, const FRow<V, float>& S, const FRow<V, float>& C,
                                const FRow<V, float>& N) {
                float ap[V], dv[V], rv[V];
                stencil_row<V>(S, C, N, wk.lane, ap);
#pragma unroll
                for (int q = 0; q < V; ++q) {
                  dv[q] = first ? __fmul_rn(am, C.f[q]) : fmx(am, C.f[q], dd.d[q]);
                  rv[q] = quantize<TR>(fmx(-am, ap[q], dd.r[q]));
                }
                acc_dot<V>(acc, j, rv, rv, nval);
                if constexpr (kPR) acc_dot<V>(aro, j, rv, dd.r, nval);
                store_row<V>(a.d, j, xl, c.nx, dv);
                store_row<V>(a.r, j, xl, c.nx, rv);
              };
              march<V, float, D>(y0, y1, wk.rev(), field, load, finish);
            }
          }
          ++wk.pc;
          constexpr int NR = kPR ? 2 : 1;
          double v[NR], o[NR];
          v[0] = acc.value();
          if constexpr (kPR) v[NR - 1] = aro.value();
          if (!tm.template reduce<NR>(v, o, red)) { aborted = true; goto done; }
          const double gnew = o[0];
          ++k;
          ++total;
          if (!isfinite(gnew)) { status = LAP5CG_ERR_BREAKDOWN; goto done; }
          beta = (kPR ? gnew - o[NR - 1] : gnew) / gamma;
          gamma = gnew;
          cur ^= 1;
        }
      }
      have_d = (k > 0);
    }
    ++outer;
  }
done:
  if (ring.S > 0) ring.teardown();
  write_info(c, tm.rank(), status, aborted, total, outer, rr, bb, relres_true);
}

}  // namespace lap5
