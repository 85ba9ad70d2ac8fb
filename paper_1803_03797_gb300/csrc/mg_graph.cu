// mg_graph.cu -- the multigrid-preconditioned CG (Algorithm 1 with M^-1 one
// V-cycle; precisions MG_F32 / MG_F64, classic variant) as a CUDA graph: one
// ordinary kernel per pass, each at the occupancy its own registers allow,
// and the PCG iterations looped on the device by a WHILE conditional node
// whose condition the convergence check sets.  Scalars stay in device memory;
// there is no host round trip per iteration and no grid barrier (the kernel
// boundaries order the passes).
//
// The persistent kernel of mg.cu runs every pass inside one launch at 16 warps
// an SM (its register budget, with the V-cycle driver and the PCG state live)
// and a grid barrier between passes, where the level passes are latency-bound.
// Same arithmetic and operation order per point as there; the dot products are
// summed per block, then over blocks in a fixed order.
//
// The host replays the V-cycle's pass sequence (Vcycle::run in mg_kernels.cuh:
// which buffer each pass reads and writes, the march direction) into one
// kernel node per pass; the levels of at most kMgCtaPoints points run in one
// single-CTA kernel node.  Instantiated graphs are cached per call signature
// (device, shape, workspace, V-cycle options); a small kernel writes each
// call's b, x, info, history, tol and maxit into the workspace before the
// cached graph is launched.
#include <mutex>
#include <vector>

#include "mg_kernels.cuh"

namespace lap5 {

constexpr int kGmThreads = 256;
constexpr int kGmMaxBlocks = 4096;  // partial-sum slots

// Solve state in device memory (the workspace's control block).
struct GmScal {
  double bb, thr, rr, gamma, alpha, beta;
  int iters, status, stop, cur, zero_x, pad;
};

// Per-call arguments, written by k_gm_bind before each graph launch, so that
// one instantiated graph serves every right-hand side, solution, tolerance and
// iteration limit on the same shape and workspace.
struct GmBind {
  const double* b;
  double* x;
  lap5cg_info* info;
  double* history;
  double tol;
  int maxit, pad;
};

__global__ void k_gm_bind(GmBind* bd, const double* b, double* x, lap5cg_info* info, double* history, double tol,
                          int maxit) {
  if (threadIdx.x == 0 && blockIdx.x == 0) *bd = GmBind{b, x, info, history, tol, maxit, 0};
}

enum { GP_JAC = 0, GP_JAC_DOT, GP_RES, GP_RESTRICT, GP_PROLONG };

// Block-wide sums of NV per-thread values into part[blockIdx.x * 2 + k].
template <int NV>
__device__ __forceinline__ void gm_partials(const double (&v)[NV], double* part) {
  __shared__ double sred[32][2];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int k = 0; k < NV; ++k) {
    double s = v[k];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) sred[warp][k] = s;
  }
  __syncthreads();
  if (warp == 0) {
#pragma unroll
    for (int k = 0; k < NV; ++k) {
      double s = lane < nw ? sred[lane][k] : 0.0;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
      if (lane == 0) part[blockIdx.x * 2 + k] = s;
    }
  }
}

// One-block sum of part[b * 2 + k] over nb blocks (fixed order); every thread
// gets the total.
__device__ __forceinline__ double gm_total(const double* part, int nb, int k) {
  __shared__ double sw[32];
  __shared__ double total;
  double s = 0.0;
  for (int b = threadIdx.x; b < nb; b += blockDim.x) s += part[b * 2 + k];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (lane == 0) sw[warp] = s;
  __syncthreads();
  if (warp == 0) {
    double t = lane < nw ? sw[lane] : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    if (lane == 0) total = t;
  }
  __syncthreads();
  const double r = total;
  __syncthreads();
  return r;
}

__device__ __forceinline__ Sched gm_sched(int rev) {
  const int wpc = blockDim.x >> 5;
  return Sched{(int)blockIdx.x * wpc + (int)(threadIdx.x >> 5), (int)gridDim.x * wpc, (int)(threadIdx.x & 31),
               rev != 0};
}

// One V-cycle pass on a big level (see the GP_ kinds); in / out are the
// level's buffers, Lc the next coarser level (restriction, prolongation).
template <class TM>
__global__ void __launch_bounds__(kGmThreads) k_gm_pass(const GmScal* sc, double* part, MgLevel<TM> L,
                                                         MgLevel<TM> Lc, int kind, int rev, const TM* in, TM* out,
                                                         Grid<const double> r) {
  if (sc->stop) return;  // the solve has ended (uniform over the grid)
  const Sched s = gm_sched(rev);
  Acc64 acc;
  switch (kind) {
    case GP_JAC: mg_stencil_pass<TM, true, false>(s, L, in, out, r, acc); break;
    case GP_JAC_DOT: {
      mg_stencil_pass<TM, true, true>(s, L, in, out, r, acc);
      const double v[1] = {acc.value()};
      gm_partials<1>(v, part);
      break;
    }
    case GP_RES: mg_stencil_pass<TM, false, false>(s, L, in, out, r, acc); break;
    case GP_RESTRICT: mg_restrict(s, L, in, Lc); break;      // in: the level's residual
    default: mg_prolong(s, L, out, Lc, in); break;            // out (fine iterate) += P in (coarse iterate)
  }
}

// The levels of at most kMgCtaPoints points, from `first` (whose b and first
// sweep the restriction wrote) down to the coarsest and back, on one CTA.
template <class TM>
struct GmLevels {
  MgLevel<TM> lv[kMgMaxLevels];
};

template <class TM>
__global__ void __launch_bounds__(512) k_gm_small(const GmScal* sc, GmLevels<TM> levels, int nlev, int first, int nu,
                                                  int nu_c) {
  if (sc->stop) return;
  __shared__ double red[kRedDoubles];
  __shared__ MgLevel<TM> lv[kMgMaxLevels];
  if (threadIdx.x < kMgMaxLevels) lv[threadIdx.x] = levels.lv[threadIdx.x];
  __syncthreads();
  GridTeam tm{nullptr, 0, 0ull};  // never synchronised: every level here is CTA-local
  const int wpc = blockDim.x >> 5;
  const Sched cta{(int)(threadIdx.x >> 5), wpc, (int)(threadIdx.x & 31), false};
  Vcycle<TM> vc{nlev, first, nu, nu_c, lv, tm, red, cta, cta, Grid<const double>{nullptr, 0}, nullptr, {}, true,
                false, 0u};
  vc.cur[first] = 0;
  for (int l = first; l < nlev - 1; ++l) vc.down(l);
  vc.sweeps(nlev - 1, nu_c, false);
  for (int l = nlev - 2; l >= first; --l) vc.up(l);
}

// r = b - A x, level 0: b = r (rounded to TM), u = c b; partials (b, b), (r, r).
template <class TM>
__global__ void __launch_bounds__(kGmThreads) k_gm_init(const GmBind* bd, double* part, int nx, int ny, int ld,
                                                         Grid<double> r, MgLevel<TM> L0) {
  constexpr int V = 2;
  const Grid<const double> b{bd->b, ld};
  const Grid<double> x{bd->x, ld};
  const Sched s = gm_sched(0);
  const Units un = make_units(nx, ny, V, s.nw, 2);
  const Grid<TM> g0b{L0.b, L0.ld}, g0u{L0.u, L0.ld};
  const TM cm = (TM)kMgC;
  Acc64 abb, arr;
  struct D { double b[V]; };
  for (int u = s.w; u < un.nunits; u += s.nw) {
    int st, y0, y1;
    unit_bounds(un, u, ny, st, y0, y1);
    const int xs = st * 32 * V, xl = Lanes<V>::first(xs, s.lane);
    const int nval = nx - xl;
    auto field = [&](int j, FRow<V, double>& f) { field_plain<V>(x, nx, ny, j, xl, xs, s.lane, f); };
    auto load = [&](int j, D& d) { load_row<V>(b, j, xl, nx, d.b); };
    auto finish = [&](int j, const D& d, const FRow<V, double>& S, const FRow<V, double>& C,
                      const FRow<V, double>& N) {
      double ax[V], rv[V];
      TM rb[V], ru[V];
      stencil_row<V>(S, C, N, s.lane, ax);
#pragma unroll
      for (int k = 0; k < V; ++k) {
        rv[k] = d.b[k] - ax[k];
        rb[k] = (TM)rv[k];
        ru[k] = cm * rb[k];
      }
      acc_dot<V>(abb, j, d.b, d.b, nval);
      acc_dot<V>(arr, j, rv, rv, nval);
      store_row<V>(r, j, xl, nx, rv);
      store_row<V>(g0b, j, xl, nx, rb);
      store_row<V>(g0u, j, xl, nx, ru);
    };
    march<V, double, D>(y0, y1, false, field, load, finish);
  }
  const double v[2] = {abb.value(), arr.value()};
  gm_partials<2>(v, part);
}

// (b, b), (r, r) -> threshold, status; the loop's condition.
__global__ void __launch_bounds__(256) k_gm_start(GmScal* sc, const GmBind* bd, const double* part, int nb,
                                                  cudaGraphConditionalHandle h) {
  const double tol = bd->tol;
  const int maxit = bd->maxit;
  double* history = bd->history;
  const double bb = gm_total(part, nb, 0), rr = gm_total(part, nb, 1);
  if (threadIdx.x != 0) return;
  GmScal s = {};
  s.bb = bb;
  s.rr = rr;
  s.thr = tol > 0.0 ? tol * tol * bb : 0.0;
  s.status = LAP5CG_NOT_CONVERGED;
  s.stop = 1;
  if (!isfinite(bb)) {
    s.status = LAP5CG_ERR_NONFINITE;
  } else if (bb == 0.0) {
    s.status = LAP5CG_OK;
    s.zero_x = 1;
    s.rr = 0.0;
  } else {
    if (history) history[0] = sqrt(rr / bb);
    if (!isfinite(rr)) s.status = LAP5CG_ERR_NONFINITE;
    else if (rr <= s.thr) s.status = LAP5CG_OK;
    else if (maxit > 0) s.stop = 0;
  }
  *sc = s;
  cudaGraphSetConditional(h, s.stop ? 0u : 1u);
}

// (r, z) -> beta, gamma (breakdown if not positive).
__global__ void __launch_bounds__(256) k_gm_rz(GmScal* sc, const double* part, int nb) {
  if (sc->stop) return;
  const double rz = gm_total(part, nb, 0);
  if (threadIdx.x != 0) return;
  if (!(rz > 0.0) || !isfinite(rz)) {
    sc->status = LAP5CG_ERR_BREAKDOWN;
    sc->stop = 1;
    return;
  }
  sc->beta = (sc->iters == 0) ? 0.0 : rz / sc->gamma;
  sc->gamma = rz;
}

// p = z + beta p (halo included), q = A p, partial (p, q).
template <class TM>
__global__ void __launch_bounds__(kGmThreads) k_gm_pq(const GmScal* sc, double* part, int nx, int ny,
                                                       Grid<double> p0, Grid<double> p1, Grid<double> q,
                                                       MgLevel<TM> L0, int zbuf, int rev) {
  if (sc->stop) return;
  constexpr int V = 2;
  const Sched s = gm_sched(rev);
  const Units un = make_units(nx, ny, V, s.nw, 2);
  const double beta = sc->beta;
  const bool first = (sc->iters == 0);
  const Grid<double> pold = sc->cur ? p1 : p0;
  const Grid<double> pnew = sc->cur ? p0 : p1;
  const Grid<const TM> gz{zbuf ? L0.v : L0.u, L0.ld};
  Acc64 apq;
  struct D { int dummy; };
  for (int u = s.w; u < un.nunits; u += s.nw) {
    int st, y0, y1;
    unit_bounds(un, u, ny, st, y0, y1);
    const int xs = st * 32 * V, xl = Lanes<V>::first(xs, s.lane);
    const int nval = nx - xl;
    auto zone = [&](int j, int xx) -> double { return (xx < 0 || xx >= nx) ? 0.0 : (double)gz.row(j)[xx]; };
    auto pone = [&](int j, int xx) -> double { return (xx < 0 || xx >= nx) ? 0.0 : pold.row(j)[xx]; };
    auto field = [&](int j, FRow<V, double>& f) {
      if (j < 0 || j >= ny) { f.zero(); return; }
      TM zt[V];
      load_row<V>(gz, j, xl, nx, zt);
      if (first) {
#pragma unroll
        for (int k = 0; k < V; ++k) f.f[k] = (double)zt[k];
        f.hl = (s.lane == 0) ? zone(j, xs - 1) : 0.0;
        f.hr = (s.lane == 31) ? zone(j, xs + 32 * V) : 0.0;
      } else {
        double pv[V];
        load_row<V>(pold, j, xl, nx, pv);
#pragma unroll
        for (int k = 0; k < V; ++k) f.f[k] = __fma_rn(beta, pv[k], (double)zt[k]);
        f.hl = (s.lane == 0) ? __fma_rn(beta, pone(j, xs - 1), zone(j, xs - 1)) : 0.0;
        f.hr = (s.lane == 31) ? __fma_rn(beta, pone(j, xs + 32 * V), zone(j, xs + 32 * V)) : 0.0;
      }
    };
    auto load = [&](int, D&) {};
    auto finish = [&](int j, const D&, const FRow<V, double>& S, const FRow<V, double>& C, const FRow<V, double>& N) {
      double qv[V];
      stencil_row<V>(S, C, N, s.lane, qv);
      store_row<V>(pnew, j, xl, nx, C.f);
      store_row<V>(q, j, xl, nx, qv);
      acc_dot<V>(apq, j, C.f, qv, nval);
    };
    march<V, double, D>(y0, y1, s.rev, field, load, finish);
  }
  const double v[1] = {apq.value()};
  gm_partials<1>(v, part);
}

// (p, q) -> alpha (breakdown if not positive); the new p becomes current.
__global__ void __launch_bounds__(256) k_gm_alpha(GmScal* sc, const double* part, int nb) {
  if (sc->stop) return;
  const double pq = gm_total(part, nb, 0);
  if (threadIdx.x != 0) return;
  if (!(pq > 0.0) || !isfinite(pq)) {
    sc->status = LAP5CG_ERR_BREAKDOWN;
    sc->stop = 1;
    return;
  }
  sc->alpha = sc->gamma / pq;
  sc->cur ^= 1;
}

// x += alpha p, r -= alpha q, partial (r, r); level 0: b = r, u = c b.
template <class TM>
__global__ void __launch_bounds__(kGmThreads) k_gm_xr(const GmScal* sc, const GmBind* bd, double* part, int nx,
                                                       int ny, int ld, Grid<double> r, Grid<double> p0,
                                                       Grid<double> p1, Grid<double> q, MgLevel<TM> L0, int rev) {
  if (sc->stop) return;
  constexpr int V = 2;
  const Grid<double> x{bd->x, ld};
  const Sched s = gm_sched(rev);
  const Units un = make_units(nx, ny, V, s.nw, 2);
  const double alpha = sc->alpha;
  const Grid<double> p = sc->cur ? p1 : p0;  // the p formed by k_gm_pq (cur was flipped since)
  const Grid<TM> g0b{L0.b, L0.ld}, g0u{L0.u, L0.ld};
  const TM cm = (TM)kMgC;
  Acc64 arr;
  struct D { double x[V], r[V], p[V], q[V]; };
  for (int u = s.w; u < un.nunits; u += s.nw) {
    int st, y0, y1;
    unit_bounds(un, u, ny, st, y0, y1);
    const int xl = Lanes<V>::first(st * 32 * V, s.lane);
    const int nval = nx - xl;
    auto load = [&](int j, D& d) {
      load_row<V>(x, j, xl, nx, d.x);
      load_row<V>(r, j, xl, nx, d.r);
      load_row<V>(p, j, xl, nx, d.p);
      load_row<V>(q, j, xl, nx, d.q);
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
      store_row<V>(x, j, xl, nx, xv);
      store_row<V>(r, j, xl, nx, rv);
      store_row<V>(g0b, j, xl, nx, rb);
      store_row<V>(g0u, j, xl, nx, ru);
    };
    stream_rows<D>(y0, y1, s.rev, load, finish);
  }
  const double v[1] = {arr.value()};
  gm_partials<1>(v, part);
}

// (r, r) -> iteration count, history, convergence; the loop's condition.
__global__ void __launch_bounds__(256) k_gm_check(GmScal* sc, const GmBind* bd, const double* part, int nb,
                                                  cudaGraphConditionalHandle h) {
  if (sc->stop) {
    if (threadIdx.x == 0) cudaGraphSetConditional(h, 0u);
    return;
  }
  const double rr = gm_total(part, nb, 0);
  if (threadIdx.x != 0) return;
  const int maxit = bd->maxit;
  double* history = bd->history;
  GmScal s = *sc;
  s.rr = rr;
  s.iters += 1;
  if (history) history[s.iters] = sqrt(rr / s.bb);
  if (!isfinite(rr)) {
    s.status = LAP5CG_ERR_NONFINITE;
    s.stop = 1;
  } else if (rr <= s.thr) {
    s.status = LAP5CG_OK;
    s.stop = 1;
  } else if (s.iters >= maxit) {
    s.stop = 1;
  }
  *sc = s;
  cudaGraphSetConditional(h, s.stop ? 0u : 1u);
}

// After the loop: x = 0 for b = 0; partial (r, r) of the true residual b - A x.
__global__ void __launch_bounds__(kGmThreads) k_gm_true(const GmScal* sc, const GmBind* bd, double* part, int nx,
                                                         int ny, int ld, int true_res) {
  constexpr int V = 2;
  const Grid<const double> b{bd->b, ld};
  const Grid<double> x{bd->x, ld};
  const Sched s = gm_sched(0);
  const Units un = make_units(nx, ny, V, s.nw, 2);
  if (sc->zero_x) {
    for (int u = s.w; u < un.nunits; u += s.nw) {
      int st, y0, y1;
      unit_bounds(un, u, ny, st, y0, y1);
      const int xl = Lanes<V>::first(st * 32 * V, s.lane);
      const double z[V] = {0.0, 0.0};
      for (int j = y0; j < y1; ++j) store_row<V>(x, j, xl, nx, z);
    }
    return;
  }
  if (!true_res) return;
  Acc64 arr;
  struct D { double b[V]; };
  for (int u = s.w; u < un.nunits; u += s.nw) {
    int st, y0, y1;
    unit_bounds(un, u, ny, st, y0, y1);
    const int xs = st * 32 * V, xl = Lanes<V>::first(xs, s.lane);
    const int nval = nx - xl;
    auto field = [&](int j, FRow<V, double>& f) { field_plain<V>(x, nx, ny, j, xl, xs, s.lane, f); };
    auto load = [&](int j, D& d) { load_row<V>(b, j, xl, nx, d.b); };
    auto finish = [&](int j, const D& d, const FRow<V, double>& S, const FRow<V, double>& C,
                      const FRow<V, double>& N) {
      double ax[V], rv[V];
      stencil_row<V>(S, C, N, s.lane, ax);
#pragma unroll
      for (int k = 0; k < V; ++k) rv[k] = d.b[k] - ax[k];
      acc_dot<V>(arr, j, rv, rv, nval);
    };
    march<V, double, D>(y0, y1, false, field, load, finish);
  }
  const double v[1] = {arr.value()};
  gm_partials<1>(v, part);
}

__global__ void __launch_bounds__(256) k_gm_finish(const GmScal* sc, const GmBind* bd, const double* part, int nb,
                                                   int true_res) {
  const bool have = true_res && !sc->zero_x && isfinite(sc->bb) && sc->bb > 0.0;
  const double rt = have ? gm_total(part, nb, 0) : 0.0;
  if (threadIdx.x != 0) return;
  lap5cg_info inf;
  inf.status = sc->status;
  inf.iters = sc->iters;
  inf.outer_iters = 0;
  inf.pad = 0;
  inf.relres_recursive = (sc->bb > 0.0 && isfinite(sc->bb)) ? sqrt(sc->rr / sc->bb) : 0.0;
  inf.relres_true = sc->zero_x ? 0.0 : (have ? sqrt(rt / sc->bb) : nan(""));
  *bd->info = inf;
}

// ---------------------------------------------------------------------------
// Host: the pass list, the graph, the cache.
// ---------------------------------------------------------------------------
template <class TM>
struct GmPassRec {
  int kind, level, rev;
  const TM* in;
  TM* out;
};

// The V-cycle's passes on the big levels as Vcycle::run executes them (buffer
// parities and march directions), with the single-CTA levels as one entry
// (kind -1).  Returns the buffer that holds level 0's result (M^-1 r).
template <class TM>
static int gm_pass_list(const PcgArgs<TM>& a, std::vector<GmPassRec<TM>>& out) {
  const int L = a.nlev, nu = a.nu;
  int cur[kMgMaxLevels] = {0};
  unsigned pc = 0;
  auto it = [&](int l) -> TM* { return cur[l] ? a.lv[l].v : a.lv[l].u; };
  auto other = [&](int l) -> TM* { return cur[l] ? a.lv[l].u : a.lv[l].v; };
  auto jac = [&](int l, bool last) {
    out.push_back({last ? GP_JAC_DOT : GP_JAC, l, (int)(pc++ & 1u), it(l), other(l)});
    cur[l] ^= 1;
  };
  auto sweeps = [&](int l, int n, bool final0) {
    for (int k = 1; k < n; ++k) jac(l, final0 && l == 0 && k == n - 1);
  };
  const int big_end = a.lsmall < L - 1 ? a.lsmall : L - 1;
  for (int l = 0; l < big_end; ++l) {  // down: pre-smoothing, residual, restriction
    sweeps(l, nu, false);
    out.push_back({GP_RES, l, (int)(pc++ & 1u), it(l), other(l)});
    out.push_back({GP_RESTRICT, l, (int)(pc++ & 1u), other(l), nullptr});
    cur[l + 1] = 0;
  }
  if (a.lsmall >= L) {
    sweeps(L - 1, a.nu_c, false);
  } else {
    out.push_back({-1, big_end, 0, nullptr, nullptr});
    // the single-CTA kernel leaves level big_end's iterate after 2 nu - 1
    // sweeps (nu - 1 down, nu up), or nu_c - 1 if it is the coarsest
    const int flips = big_end < L - 1 ? 2 * nu - 1 : a.nu_c - 1;
    cur[big_end] = flips & 1;
  }
  for (int l = big_end - 1; l >= 0; --l) {  // up: prolongation, post-smoothing
    out.push_back({GP_PROLONG, l, (int)(pc++ & 1u), it(l + 1), it(l)});
    for (int k = 0; k < nu; ++k) jac(l, l == 0 && k == nu - 1);
  }
  return cur[0];
}

// What an instantiated graph bakes in: the shape, the V-cycle options and the
// workspace (b, x, info, history, tol and maxit go through GmBind).
struct GmKey {
  int dev, nx, ny, ld, ldw, true_res, nu, nu_c, levels, f32;
  const void* ws;
  bool operator==(const GmKey& o) const {
    return dev == o.dev && nx == o.nx && ny == o.ny && ld == o.ld && ldw == o.ldw && true_res == o.true_res &&
           nu == o.nu && nu_c == o.nu_c && levels == o.levels && f32 == o.f32 && ws == o.ws;
  }
};

static std::mutex g_gm_mu;
static std::vector<std::pair<GmKey, cudaGraphExec_t>> g_gm_cache;  // most recent last
constexpr size_t kGmCacheSize = 8;

static int gm_add(cudaGraph_t g, cudaGraphNode_t* prev, const void* fn, unsigned grid, unsigned block, void** args) {
  cudaKernelNodeParams kp = {};
  kp.func = const_cast<void*>(fn);
  kp.gridDim = dim3(grid);
  kp.blockDim = dim3(block);
  kp.sharedMemBytes = 0;
  kp.kernelParams = args;
  kp.extra = nullptr;
  cudaGraphNode_t n;
  if (cudaGraphAddKernelNode(&n, g, *prev ? prev : nullptr, *prev ? 1 : 0, &kp) != cudaSuccess) return LAP5CG_ERR_CUDA;
  *prev = n;
  return LAP5CG_OK;
}

static int gm_blocks(const void* fn, int threads, int sms) {
  int occ = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, threads, 0) != cudaSuccess || occ < 1) occ = 1;
  const int nb = occ * sms;
  return nb < kGmMaxBlocks ? nb : kGmMaxBlocks;
}

template <class TM>
static int gm_build(const SolvePlan& p, const PcgArgs<TM>& a, cudaGraphExec_t* exec) {
  DevProps dp;
  int rc = dev_props(&dp);
  if (rc != LAP5CG_OK) return rc;
  GmScal* sc = reinterpret_cast<GmScal*>(p.ws + 1024);
  GmBind* bd = reinterpret_cast<GmBind*>(p.ws + 2048);
  double* part = reinterpret_cast<double*>(p.ws + 4096);
  const int nx = p.nx, ny = p.ny;
  const void* f_pass = reinterpret_cast<const void*>(&k_gm_pass<TM>);
  const void* f_init = reinterpret_cast<const void*>(&k_gm_init<TM>);
  const void* f_pq = reinterpret_cast<const void*>(&k_gm_pq<TM>);
  const void* f_xr = reinterpret_cast<const void*>(&k_gm_xr<TM>);
  const void* f_true = reinterpret_cast<const void*>(&k_gm_true);
  const int nb_pass = gm_blocks(f_pass, kGmThreads, dp.sms);
  const int nb_init = gm_blocks(f_init, kGmThreads, dp.sms);
  const int nb_pq = gm_blocks(f_pq, kGmThreads, dp.sms);
  const int nb_xr = gm_blocks(f_xr, kGmThreads, dp.sms);
  const int nb_true = gm_blocks(f_true, kGmThreads, dp.sms);
  std::vector<GmPassRec<TM>> passes;
  const int zbuf = gm_pass_list<TM>(a, passes);

  cudaGraph_t g = nullptr;
  if (cudaGraphCreate(&g, 0) != cudaSuccess) return LAP5CG_ERR_CUDA;
  auto fail = [&](int code) {
    cudaGraphDestroy(g);
    return code;
  };
  cudaGraphConditionalHandle h;
  if (cudaGraphConditionalHandleCreate(&h, g, 0, cudaGraphCondAssignDefault) != cudaSuccess)
    return fail(LAP5CG_ERR_CUDA);
  cudaGraphNode_t prev = nullptr;
  int nx_ = nx, ny_ = ny, ld_ = p.ld;
  Grid<double> gr = a.r, gp0 = a.p0, gp1 = a.p1, gq = a.q;
  MgLevel<TM> L0 = a.lv[0];
  {
    void* args[] = {&bd, &part, &nx_, &ny_, &ld_, &gr, &L0};
    if ((rc = gm_add(g, &prev, f_init, nb_init, kGmThreads, args)) != LAP5CG_OK) return fail(rc);
  }
  int nbi = nb_init;
  {
    void* args[] = {&sc, &bd, &part, &nbi, &h};
    if ((rc = gm_add(g, &prev, reinterpret_cast<const void*>(&k_gm_start), 1, 256, args)) != LAP5CG_OK)
      return fail(rc);
  }
  // the loop: a WHILE node whose body is one PCG iteration
  cudaGraphNodeParams cp = {};
  cp.type = cudaGraphNodeTypeConditional;
  cp.conditional.handle = h;
  cp.conditional.type = cudaGraphCondTypeWhile;
  cp.conditional.size = 1;
  cudaGraphNode_t loop;
  if (cudaGraphAddNode(&loop, g, &prev, nullptr, 1, &cp) != cudaSuccess) return fail(LAP5CG_ERR_CUDA);
  cudaGraph_t body = cp.conditional.phGraph_out[0];
  {
    cudaGraphNode_t bp = nullptr;
    Grid<const double> grc{a.r.ptr, a.r.ld};
    for (const GmPassRec<TM>& pr : passes) {
      if (pr.kind < 0) {
        GmLevels<TM> lv;
        for (int l = 0; l < kMgMaxLevels; ++l) lv.lv[l] = a.lv[l];
        int nlev = a.nlev, first = pr.level, nu = a.nu, nu_c = a.nu_c;
        void* args[] = {&sc, &lv, &nlev, &first, &nu, &nu_c};
        if ((rc = gm_add(body, &bp, reinterpret_cast<const void*>(&k_gm_small<TM>), 1, 512, args)) != LAP5CG_OK)
          return fail(rc);
        continue;
      }
      MgLevel<TM> L = a.lv[pr.level];
      MgLevel<TM> Lc = a.lv[pr.level + 1 < a.nlev ? pr.level + 1 : pr.level];
      int kind = pr.kind, rev = pr.rev;
      const TM* in = pr.in;
      TM* out = pr.out;
      void* args[] = {&sc, &part, &L, &Lc, &kind, &rev, &in, &out, &grc};
      if ((rc = gm_add(body, &bp, f_pass, nb_pass, kGmThreads, args)) != LAP5CG_OK) return fail(rc);
    }
    int nbp = nb_pass;
    {
      void* args[] = {&sc, &part, &nbp};
      if ((rc = gm_add(body, &bp, reinterpret_cast<const void*>(&k_gm_rz), 1, 256, args)) != LAP5CG_OK)
        return fail(rc);
    }
    int zb = zbuf, rev1 = 1, rev0 = 0;
    {
      void* args[] = {&sc, &part, &nx_, &ny_, &gp0, &gp1, &gq, &L0, &zb, &rev1};
      if ((rc = gm_add(body, &bp, f_pq, nb_pq, kGmThreads, args)) != LAP5CG_OK) return fail(rc);
    }
    int nbq = nb_pq;
    {
      void* args[] = {&sc, &part, &nbq};
      if ((rc = gm_add(body, &bp, reinterpret_cast<const void*>(&k_gm_alpha), 1, 256, args)) != LAP5CG_OK)
        return fail(rc);
    }
    {
      void* args[] = {&sc, &bd, &part, &nx_, &ny_, &ld_, &gr, &gp0, &gp1, &gq, &L0, &rev0};
      if ((rc = gm_add(body, &bp, f_xr, nb_xr, kGmThreads, args)) != LAP5CG_OK) return fail(rc);
    }
    int nbx = nb_xr;
    {
      void* args[] = {&sc, &bd, &part, &nbx, &h};
      if ((rc = gm_add(body, &bp, reinterpret_cast<const void*>(&k_gm_check), 1, 256, args)) != LAP5CG_OK)
        return fail(rc);
    }
  }
  prev = loop;
  int tr = p.opts.true_residual;
  {
    void* args[] = {&sc, &bd, &part, &nx_, &ny_, &ld_, &tr};
    if ((rc = gm_add(g, &prev, f_true, nb_true, kGmThreads, args)) != LAP5CG_OK) return fail(rc);
  }
  int nbt = nb_true;
  {
    void* args[] = {&sc, &bd, &part, &nbt, &tr};
    if ((rc = gm_add(g, &prev, reinterpret_cast<const void*>(&k_gm_finish), 1, 256, args)) != LAP5CG_OK)
      return fail(rc);
  }
  const cudaError_t e = cudaGraphInstantiate(exec, g, 0);
  cudaGraphDestroy(g);
  return e == cudaSuccess ? LAP5CG_OK : LAP5CG_ERR_CUDA;
}

// Classic MG-PCG through the cached graph; *used = false when this shape
// takes the persistent kernel (the fine grid itself is a single-CTA level, or
// the stream is capturing).
template <class TM>
int solve_mg_graph(const SolvePlan& p, const PcgArgs<TM>& a, cudaStream_t st, bool* used) {
  *used = false;
  if (p.variant != LAP5CG_CLASSIC || a.lsmall < 1 || a.nlev < 2) return LAP5CG_OK;
  // a stream being captured into the caller's own graph gets the persistent
  // kernel: one kernel node, no nested conditional graph
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(st, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) return LAP5CG_OK;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return LAP5CG_ERR_CUDA;
  GmKey key{dev, p.nx, p.ny, p.ld, p.ldw, p.opts.true_residual, a.nu, a.nu_c, a.nlev, sizeof(TM) == 4 ? 1 : 0, p.ws};
  std::lock_guard<std::mutex> lock(g_gm_mu);
  cudaGraphExec_t exec = nullptr;
  for (size_t i = 0; i < g_gm_cache.size(); ++i)
    if (g_gm_cache[i].first == key) {
      exec = g_gm_cache[i].second;
      auto e = g_gm_cache[i];
      g_gm_cache.erase(g_gm_cache.begin() + (long)i);
      g_gm_cache.push_back(e);
      break;
    }
  if (!exec) {
    const int rc = gm_build<TM>(p, a, &exec);
    if (rc != LAP5CG_OK) return rc;
    if (g_gm_cache.size() >= kGmCacheSize) {
      cudaGraphExecDestroy(g_gm_cache.front().second);
      g_gm_cache.erase(g_gm_cache.begin());
    }
    g_gm_cache.push_back({key, exec});
  }
  k_gm_bind<<<1, 32, 0, st>>>(reinterpret_cast<GmBind*>(p.ws + 2048), static_cast<const double*>(p.b),
                              static_cast<double*>(p.x), p.info, p.opts.history, p.tol, p.maxit);
  if (cudaGetLastError() != cudaSuccess || cudaGraphLaunch(exec, st) != cudaSuccess) return LAP5CG_ERR_CUDA;
  *used = true;
  return LAP5CG_OK;
}

template int solve_mg_graph<float>(const SolvePlan&, const PcgArgs<float>&, cudaStream_t, bool*);
template int solve_mg_graph<double>(const SolvePlan&, const PcgArgs<double>&, cudaStream_t, bool*);

}  // namespace lap5
