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
#include "cg_launch.cuh"

namespace lap5 {

constexpr int kMgMaxLevels = 24;
constexpr int kMgCtaPoints = 16384;  // levels this small run on one CTA
constexpr double kMgC = 0.2;         // omega / 4 with omega = 4/5

template <class TM>
struct MgLevel {
  int nx, ny;    // dense grid, pitch nx
  TM *b, *u, *v;  // right-hand side and two iterate buffers
};

template <class TM>
struct PcgArgs {
  SolveCommon c;
  Grid<const double> b;
  Grid<double> x, r, p, q;
  MgLevel<TM> lv[kMgMaxLevels];
  int nlev;    // levels (>= 1); level nlev-1 is the coarsest
  int lsmall;  // first level run by CTA 0 alone (nlev: none)
  int nu, nu_c;
};

// rows over warps, columns over lanes
struct Sched {
  int w, nw, lane;
};

template <class F>
__device__ __forceinline__ void for_points(const Sched& s, int nx, int ny, F&& f) {
  for (int j = s.w; j < ny; j += s.nw)
    for (int i = s.lane; i < nx; i += 32) f(i, j);
}

template <class T>
__device__ __forceinline__ T mg_at(const T* a, int nx, int ny, int i, int j) {
  return (i < 0 || i >= nx || j < 0 || j >= ny) ? T(0) : a[(size_t)j * nx + i];
}

// (A a)(i, j) in the Sec. II-B add order
template <class T>
__device__ __forceinline__ T mg_apply(const T* a, int nx, int ny, int i, int j) {
  T acc = T(4) * a[(size_t)j * nx + i];
  acc -= mg_at(a, nx, ny, i - 1, j);
  acc -= mg_at(a, nx, ny, i + 1, j);
  acc -= mg_at(a, nx, ny, i, j - 1);
  acc -= mg_at(a, nx, ny, i, j + 1);
  return acc;
}

__device__ __forceinline__ float mg_fma(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double mg_fma(double a, double b, double c) { return __fma_rn(a, b, c); }

// out = in + c (b - A in)
template <class TM>
__device__ void mg_jacobi(const Sched& s, const MgLevel<TM>& L, const TM* in, TM* out) {
  const TM c = (TM)kMgC;
  for_points(s, L.nx, L.ny, [&](int i, int j) {
    const size_t k = (size_t)j * L.nx + i;
    out[k] = mg_fma(c, L.b[k] - mg_apply(in, L.nx, L.ny, i, j), in[k]);
  });
}

// out = b - A in
template <class TM>
__device__ void mg_residual(const Sched& s, const MgLevel<TM>& L, const TM* in, TM* out) {
  for_points(s, L.nx, L.ny, [&](int i, int j) {
    const size_t k = (size_t)j * L.nx + i;
    out[k] = L.b[k] - mg_apply(in, L.nx, L.ny, i, j);
  });
}

// C.b = P^T res (fine F), and the first sweep from zero: C.u = c C.b
template <class TM>
__device__ void mg_restrict(const Sched& s, const MgLevel<TM>& F, const TM* res, const MgLevel<TM>& C) {
  const TM c = (TM)kMgC;
  for_points(s, C.nx, C.ny, [&](int I, int J) {
    const int i = 2 * I + 1, j = 2 * J + 1;
    const TM rC = res[(size_t)j * F.nx + i];
    const TM s1 = ((mg_at(res, F.nx, F.ny, i - 1, j) + mg_at(res, F.nx, F.ny, i + 1, j)) +
                   mg_at(res, F.nx, F.ny, i, j - 1)) + mg_at(res, F.nx, F.ny, i, j + 1);
    const TM s2 = ((mg_at(res, F.nx, F.ny, i - 1, j - 1) + mg_at(res, F.nx, F.ny, i + 1, j - 1)) +
                   mg_at(res, F.nx, F.ny, i - 1, j + 1)) + mg_at(res, F.nx, F.ny, i + 1, j + 1);
    const TM bc = TM(0.25) * ((TM(4) * rC + TM(2) * s1) + s2);
    const size_t k = (size_t)J * C.nx + I;
    C.b[k] = bc;
    C.u[k] = c * bc;
  });
}

// f += P e (coarse C)
template <class TM>
__device__ void mg_prolong(const Sched& s, const MgLevel<TM>& F, TM* f, const MgLevel<TM>& C, const TM* e) {
  for_points(s, F.nx, F.ny, [&](int i, int j) {
    const int I = i >> 1, J = j >> 1;
    TM v;
    if ((i & 1) && (j & 1)) {
      v = mg_at(e, C.nx, C.ny, I, J);
    } else if (!(i & 1) && (j & 1)) {
      v = TM(0.5) * (mg_at(e, C.nx, C.ny, I - 1, J) + mg_at(e, C.nx, C.ny, I, J));
    } else if ((i & 1) && !(j & 1)) {
      v = TM(0.5) * (mg_at(e, C.nx, C.ny, I, J - 1) + mg_at(e, C.nx, C.ny, I, J));
    } else {
      v = TM(0.25) * ((mg_at(e, C.nx, C.ny, I - 1, J - 1) + mg_at(e, C.nx, C.ny, I, J - 1)) +
                      (mg_at(e, C.nx, C.ny, I - 1, J) + mg_at(e, C.nx, C.ny, I, J)));
    }
    f[(size_t)j * F.nx + i] += v;
  });
}

template <class TM>
struct Vcycle {
  int nlev, lsmall, nu, nu_c;  // as in PcgArgs
  const MgLevel<TM>* lv;       // the level descriptors, staged in shared memory
  GridTeam& tm;
  double* red;
  Sched grid, cta;
  int cur[kMgMaxLevels];  // 0: the level's iterate is in u, 1: in v
  bool exec;              // this CTA runs the passes it meets (small levels: CTA 0 only)

  __device__ TM* it(int l) const { return cur[l] ? lv[l].v : lv[l].u; }
  __device__ TM* other(int l) const { return cur[l] ? lv[l].u : lv[l].v; }
  __device__ bool small(int l) const { return l >= lsmall; }
  __device__ const Sched& sched(int l) const { return small(l) ? cta : grid; }
  // barrier after a pass at level l: grid-wide for big levels, CTA-wide for
  // small ones (which only CTA 0 runs)
  __device__ bool sync(int l) {
    if (small(l)) {
      __syncthreads();
      return true;
    }
    return tm.sync(red);
  }
  // One pass at level l, then its barrier.  A CTA that does not run small
  // levels only follows the iterate buffers.
  template <class F>
  __device__ bool pass(int l, F&& f) {
    if (!exec) return true;
    f(sched(l));
    return sync(l);
  }
  // sweeps 2..n of damped Jacobi (the first sweep, u = c b, came with b)
  __device__ bool sweeps(int l, int n) {
    for (int k = 1; k < n; ++k) {
      if (!pass(l, [&](const Sched& s) { mg_jacobi(s, lv[l], it(l), other(l)); })) return false;
      cur[l] ^= 1;
    }
    return true;
  }
  __device__ bool down(int l) {  // pre-smoothing, residual, restriction into l+1
    if (!sweeps(l, nu)) return false;
    if (!pass(l, [&](const Sched& s) { mg_residual(s, lv[l], it(l), other(l)); })) return false;
    if (!pass(l, [&](const Sched& s) { mg_restrict(s, lv[l], other(l), lv[l + 1]); })) return false;
    cur[l + 1] = 0;
    return true;
  }
  __device__ bool up(int l) {  // prolongation from l+1, then nu post-smoothing sweeps
    if (!pass(l, [&](const Sched& s) { mg_prolong(s, lv[l], it(l), lv[l + 1], it(l + 1)); })) return false;
    for (int k = 0; k < nu; ++k) {
      if (!pass(l, [&](const Sched& s) { mg_jacobi(s, lv[l], it(l), other(l)); })) return false;
      cur[l] ^= 1;
    }
    return true;
  }
  // One V-cycle; level 0's b and u = c b are in place.  Returns false when
  // the solve must stop (abort or barrier timeout).
  __device__ bool run() {
    const int L = nlev;
    cur[0] = 0;
    const int big_end = min(lsmall, L - 1);  // levels [0, big_end) restrict grid-wide
    exec = true;
    for (int l = 0; l < big_end; ++l)
      if (!down(l)) return false;
    if (lsmall >= L) {  // the coarsest level is big
      if (!sweeps(L - 1, nu_c)) return false;
    } else {
      exec = blockIdx.x == 0;  // CTA 0 alone; the others follow the buffers
      for (int l = big_end; l < L - 1; ++l) down(l);
      sweeps(L - 1, nu_c);
      for (int l = L - 2; l >= big_end; --l) up(l);
      exec = true;
      if (!tm.sync(red)) return false;  // publishes CTA 0's levels
    }
    for (int l = big_end - 1; l >= 0; --l)
      if (!up(l)) return false;
    return true;
  }
};

template <class TM>
__device__ __forceinline__ void pcg_solve(const PcgArgs<TM>& a, const MgLevel<TM>* lv, GridTeam& tm, double* red) {
  const SolveCommon& c = a.c;
  const int lane = threadIdx.x & 31;
  const int wpc = blockDim.x >> 5;
  const Sched grid{(int)blockIdx.x * wpc + (int)(threadIdx.x >> 5), (int)gridDim.x * wpc, lane};
  const Sched cta{(int)(threadIdx.x >> 5), wpc, lane};
  const MgLevel<TM> L0 = lv[0];
  const TM cm = (TM)kMgC;
  int status = LAP5CG_NOT_CONVERGED, iters = 0;
  double bb = 0.0, rr = 0.0, gamma = 0.0, relres_true = nan("");
  bool aborted = false;
  Vcycle<TM> vc{a.nlev, a.lsmall, a.nu, a.nu_c, lv, tm, red, grid, cta, {}, true};

  // the iterate of level 0 after a V-cycle, as binary64 (z = M^-1 r)
  auto z_at = [&](size_t k) -> double { return (double)vc.it(0)[k]; };

  {  // r = b - A x; (b, b), (r, r); level 0: b = r, u = c b
    Acc64 abb, arr;
    for_points(grid, c.nx, c.ny, [&](int i, int j) {
      const double* xr = a.x.ptr;
      const int ld = a.x.ld;
      auto X = [&](int ii, int jj) -> double {
        return (ii < 0 || ii >= c.nx || jj < 0 || jj >= c.ny) ? 0.0 : xr[(size_t)jj * ld + ii];
      };
      double acc = 4.0 * X(i, j);
      acc -= X(i - 1, j);
      acc -= X(i + 1, j);
      acc -= X(i, j - 1);
      acc -= X(i, j + 1);
      const double bv = a.b.row(j)[i], rv = bv - acc;
      a.r.row(j)[i] = rv;
      abb.add(bv, bv);
      arr.add(rv, rv);
      const size_t k = (size_t)j * L0.nx + i;
      L0.b[k] = (TM)rv;
      L0.u[k] = cm * (TM)rv;
    });
    double v[2] = {abb.value(), arr.value()}, o[2];
    if (!tm.template reduce<2>(v, o, red)) { aborted = true; goto done; }
    bb = o[0];
    rr = o[1];
  }
  if (!isfinite(bb)) { status = LAP5CG_ERR_NONFINITE; goto done; }
  if (bb == 0.0) {
    for_points(grid, c.nx, c.ny, [&](int i, int j) { a.x.row(j)[i] = 0.0; });
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
    double beta = 0.0;
    for (;;) {
      // z = M^-1 r, gamma_new = (r, z)
      if (!vc.run()) { aborted = true; goto done; }
      {
        Acc64 arz;
        for_points(grid, c.nx, c.ny, [&](int i, int j) {
          arz.add(a.r.row(j)[i], z_at((size_t)j * L0.nx + i));
        });
        double v[1] = {arz.value()}, o[1];
        if (!tm.template reduce<1>(v, o, red)) { aborted = true; goto done; }
        if (!(o[0] > 0.0) || !isfinite(o[0])) { status = LAP5CG_ERR_BREAKDOWN; goto truecheck; }
        beta = (iters == 0) ? 0.0 : o[0] / gamma;
        gamma = o[0];
      }
      // p = z + beta p
      for_points(grid, c.nx, c.ny, [&](int i, int j) {
        double* pr = a.p.row(j) + i;
        const double zv = z_at((size_t)j * L0.nx + i);
        *pr = (iters == 0) ? zv : __fma_rn(beta, *pr, zv);
      });
      if (!tm.sync(red)) { aborted = true; goto done; }
      // q = A p, (p, q)
      double alpha;
      {
        Acc64 apq;
        for_points(grid, c.nx, c.ny, [&](int i, int j) {
          const double* pp = a.p.ptr;
          const int ld = a.p.ld;
          auto P = [&](int ii, int jj) -> double {
            return (ii < 0 || ii >= c.nx || jj < 0 || jj >= c.ny) ? 0.0 : pp[(size_t)jj * ld + ii];
          };
          double acc = 4.0 * P(i, j);
          acc -= P(i - 1, j);
          acc -= P(i + 1, j);
          acc -= P(i, j - 1);
          acc -= P(i, j + 1);
          a.q.row(j)[i] = acc;
          apq.add(P(i, j), acc);
        });
        double v[1] = {apq.value()}, o[1];
        if (!tm.template reduce<1>(v, o, red)) { aborted = true; goto done; }
        if (!(o[0] > 0.0) || !isfinite(o[0])) { status = LAP5CG_ERR_BREAKDOWN; goto truecheck; }
        alpha = gamma / o[0];
      }
      // x += alpha p, r -= alpha q, (r, r); level 0: b = r, u = c b
      {
        Acc64 arr;
        const TM cmm = cm;
        for_points(grid, c.nx, c.ny, [&](int i, int j) {
          double* xr = a.x.row(j) + i;
          double* rp = a.r.row(j) + i;
          const double pv = a.p.row(j)[i], qv = a.q.row(j)[i];
          *xr = __fma_rn(alpha, pv, *xr);
          const double rv = __fma_rn(-alpha, qv, *rp);
          *rp = rv;
          arr.add(rv, rv);
          const size_t k = (size_t)j * L0.nx + i;
          L0.b[k] = (TM)rv;
          L0.u[k] = cmm * (TM)rv;
        });
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
    Acc64 arr;
    for_points(grid, c.nx, c.ny, [&](int i, int j) {
      const double* xr = a.x.ptr;
      const int ld = a.x.ld;
      auto X = [&](int ii, int jj) -> double {
        return (ii < 0 || ii >= c.nx || jj < 0 || jj >= c.ny) ? 0.0 : xr[(size_t)jj * ld + ii];
      };
      double acc = 4.0 * X(i, j);
      acc -= X(i - 1, j);
      acc -= X(i + 1, j);
      acc -= X(i, j - 1);
      acc -= X(i, j + 1);
      const double rv = a.b.row(j)[i] - acc;
      arr.add(rv, rv);
    });
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

template <class TM>
static size_t mg_level_bytes(int nx, int ny) {
  int lnx[kMgMaxLevels], lny[kMgMaxLevels];
  const int L = mg_levels(nx, ny, 0, lnx, lny);
  size_t s = 0;
  for (int l = 0; l < L; ++l) s += 3 * align_up((size_t)lnx[l] * (size_t)lny[l] * sizeof(TM), kAlign);
  return s;
}

size_t ws_bytes_mg(int nx, int ny, int ldw, int variant, int precision) {
  if (variant != LAP5CG_CLASSIC) return 0;  // the outer solver is Algorithm 1
  const size_t vec = align_up((size_t)ny * (size_t)ldw * sizeof(double), kAlign);
  const size_t lv = precision == LAP5CG_PREC_MG_F32 ? mg_level_bytes<float>(nx, ny) : mg_level_bytes<double>(nx, ny);
  return kCtlBytes + 3 * vec + lv;
}

template <class TM>
static int solve_mg_t(const SolvePlan& p, cudaStream_t st) {
  const size_t vec = align_up((size_t)p.ny * (size_t)p.ldw * sizeof(double), kAlign);
  unsigned char* base = p.ws + kCtlBytes;
  if (cudaMemsetAsync(p.ws, 0, 256, st) != cudaSuccess) return LAP5CG_ERR_CUDA;
  PcgArgs<TM> a;
  int lnx[kMgMaxLevels], lny[kMgMaxLevels];
  a.nlev = mg_levels(p.nx, p.ny, p.opts.mg_levels, lnx, lny);
  unsigned char* lv = base + 3 * vec;
  a.lsmall = a.nlev;
  for (int l = 0; l < a.nlev; ++l) {
    const size_t bytes = align_up((size_t)lnx[l] * (size_t)lny[l] * sizeof(TM), kAlign);
    a.lv[l].nx = lnx[l];
    a.lv[l].ny = lny[l];
    a.lv[l].b = reinterpret_cast<TM*>(lv);
    a.lv[l].u = reinterpret_cast<TM*>(lv + bytes);
    a.lv[l].v = reinterpret_cast<TM*>(lv + 2 * bytes);
    lv += 3 * bytes;
    if (a.lsmall == a.nlev && (long long)lnx[l] * lny[l] <= kMgCtaPoints) a.lsmall = l;
  }
  a.nu = p.opts.mg_nu > 0 ? p.opts.mg_nu : 2;
  a.nu_c = p.opts.mg_coarse_sweeps > 0 ? p.opts.mg_coarse_sweeps : 8;
  LaunchCfg cfg;
  const void* fn = reinterpret_cast<const void*>(&k_pcg<TM>);
  lap5cg_opts o = p.opts;
  if (o.warps_per_cta <= 0) o.warps_per_cta = 8;  // a wider CTA 0 for the small levels
  int rc = plan_units(fn, p.nx, p.ny, 2, o, 0, &cfg);
  if (rc != LAP5CG_OK) return rc;
  RingGeom rg{0, 0, 0};
  a.c = make_common(p, cfg, rg);
  a.b = Grid<const double>{static_cast<const double*>(p.b), p.ld};
  a.x = Grid<double>{static_cast<double*>(p.x), p.ld};
  a.r = Grid<double>{reinterpret_cast<double*>(base), p.ldw};
  a.p = Grid<double>{reinterpret_cast<double*>(base + vec), p.ldw};
  a.q = Grid<double>{reinterpret_cast<double*>(base + 2 * vec), p.ldw};
  void* args[] = {&a};
  return cooperative_launch(fn, cfg, args, st, rg);
}

int solve_mg(const SolvePlan& p, cudaStream_t st) {
  if (p.variant != LAP5CG_CLASSIC) return LAP5CG_ERR_UNSUPPORTED;
  if (p.precision == LAP5CG_PREC_MG_F32) return solve_mg_t<float>(p, st);
  if (p.precision == LAP5CG_PREC_MG_F64) return solve_mg_t<double>(p, st);
  return LAP5CG_ERR_INVALID_ARG;
}

}  // namespace lap5
