// mg_graph.cu -- the multigrid-preconditioned CG (Algorithm 1 with M^-1 one
// V-cycle; precisions MG_F32 / MG_F64, classic variant) as a CUDA graph: one
// ordinary kernel per pass (or per fused group of passes: a level's descent,
// prolongation with the first post-smoothing sweep, level 0's last sweep with
// (r, z)), each at the occupancy its own registers allow,
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
// (device, shape, workspace, V-cycle options; lap5cg_release_graphs frees
// them all); a small kernel writes each call's b, x, info, history, tol and
// maxit into the workspace before the cached graph is launched.
#include <mutex>
#include <vector>

#include "mg_kernels.cuh"

namespace lap5 {

constexpr int kGmThreads = 256;
constexpr int kGmMaxBlocks = 4096;  // partial-sum slots

// Solve state in device memory (the workspace's control block).
struct GmScal {
  double bb, thr, rr, gamma, alpha, beta;
  int iters, status, stop, cur, zero_x;
  int xpend;  // x += alpha p of the last x, r pass is still to be applied (k_gm_pq or k_gm_xfinal)
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

enum { GP_JAC = 0, GP_JAC_DOT, GP_RES, GP_RESTRICT, GP_PROLONG, GP_RES_RESTRICT, GP_PROLONG_JAC, GP_JAC_RES_RESTRICT };

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

// Restriction (GP_RESTRICT: Lc.b = P^T in, in the level's residual) or
// prolongation (GP_PROLONG: out, the level's iterate, += P in, in the coarser
// level's iterate) on a big level, with the row march.
template <class TM>
__global__ void __launch_bounds__(kGmThreads) k_gm_pass(const GmScal* sc, MgLevel<TM> L, MgLevel<TM> Lc, int kind,
                                                         int rev, const TM* in, TM* out) {
  if (sc->stop) return;  // the solve has ended (uniform over the grid)
  const Sched s = gm_sched(rev);
  if (kind == GP_RESTRICT) {
    mg_restrict(s, L, in, Lc);
  } else {
    mg_prolong(s, L, out, Lc, in);
  }
}

// Jacobi sweep / residual of a big level in the layout of lap5_apply: each
// warp takes R = 2 output rows of one strip of 32 V columns and loads its R + 2
// operand rows and R right-hand-side rows before finishing the first, so no
// load waits on another (binary32: V = 8, two 16-byte groups a lane; binary64:
// V = 2).  CTAs stride over the tiles (8 warps x R rows x one strip).  Same
// arithmetic per point as mg_stencil_pass.
template <class TM> struct GmSweepVec { static constexpr int V = sizeof(TM) == 4 ? 8 : 2; };
// the (r, z) sweep: one group of columns a lane (its binary64 r rows would
// double the registers of the two-group layout)
template <class TM> struct GmDotVec { static constexpr int V = sizeof(TM) == 4 ? 4 : 2; };

// FROM_B: the input iterate is the level's first sweep from zero, c b, which is
// formed from b here (the producer of b then stores no iterate).
template <class TM, int MODE, bool FROM_B = false>
__global__ void __launch_bounds__(kGmThreads) k_gm_sweep(const GmScal* sc, double* part, MgLevel<TM> L,
                                                          const TM* in, TM* out, Grid<const double> r) {
  if (sc->stop) return;
  constexpr int V = MODE == GP_JAC_DOT ? GmDotVec<TM>::V : GmSweepVec<TM>::V, R = 2;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, wpc = blockDim.x >> 5;
  const int ns = (L.nx + 32 * V - 1) / (32 * V);
  const int band = wpc * R;
  const int ntiles = ns * ((L.ny + band - 1) / band);
  const Grid<const TM> gi{in, L.ld}, gb{L.b, L.ld};
  const Grid<TM> go{out, L.ld};
  const TM c = (TM)kMgC;
  Acc64 acc;
  for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
    const int st = t % ns;
    const int jb = (t / ns) * band + warp * R;
    if (jb >= L.ny) continue;
    const int xs = st * 32 * V, xl = Lanes<V>::first(xs, lane);
    FRow<V, TM> f[R + 2];  // operand rows jb - 1 .. jb + R
    TM bv[R][V];
#pragma unroll
    for (int k = 0; k < R + 2; ++k) {
      field_plain<V>(FROM_B ? gb : gi, L.nx, L.ny, jb - 1 + k, xl, xs, lane, f[k]);
      if constexpr (FROM_B) {
#pragma unroll
        for (int q = 0; q < V; ++q) f[k].f[q] = c * f[k].f[q];
        f[k].hl = c * f[k].hl;
        f[k].hr = c * f[k].hr;
      }
    }
#pragma unroll
    for (int k = 0; k < R; ++k) {
      if (jb + k < L.ny) {
        load_row<V>(gb, jb + k, xl, L.nx, bv[k]);
      } else {
#pragma unroll
        for (int q = 0; q < V; ++q) bv[k][q] = TM(0);
      }
    }
#pragma unroll
    for (int k = 0; k < R; ++k) {
      const int j = jb + k;
      if (j >= L.ny) break;
      TM ax[V], o[V];
      stencil_row<V>(f[k], f[k + 1], f[k + 2], lane, ax);
#pragma unroll
      for (int q = 0; q < V; ++q)
        o[q] = MODE == GP_RES ? bv[k][q] - ax[q] : mg_fma(c, bv[k][q] - ax[q], f[k + 1].f[q]);
      store_row<V>(go, j, xl, L.nx, o);
      if constexpr (MODE == GP_JAC_DOT) {
        double rv[V], zv[V];
        load_row<V>(r, j, xl, L.nx, rv);
#pragma unroll
        for (int q = 0; q < V; ++q) zv[q] = mg_widen(o[q]);
        acc_dot<V>(acc, j, rv, zv, L.nx - xl);
      }
    }
  }
  if constexpr (MODE == GP_JAC_DOT) {
    const double v[1] = {acc.value()};
    gm_partials<1>(v, part);
  }
}

// The levels of at most kMgCtaPoints points, from `first` (whose b and first
// sweep the restriction wrote) down to the coarsest and back, on one CTA with
// every level resident in its shared memory: level `first`'s b and u are
// copied in, the point-wise passes above run between CTA barriers, and level
// `first`'s final iterate is copied back to the buffer the next pass reads.
template <class TM>
struct GmLevels {
  MgLevel<TM> lv[kMgMaxLevels];
};

// Shared memory of k_gm_small: b, u, v of every level from `first` on.
template <class TM>
__host__ __device__ inline size_t gm_small_array_bytes(const MgLevel<TM>& L) {
  return align_up((size_t)L.ny * (size_t)L.ld * sizeof(TM), 16);
}
template <class TM>
static size_t gm_small_smem(const MgLevel<TM>* lv, int first, int nlev) {
  size_t s = 0;
  for (int l = first; l < nlev; ++l) s += 3 * gm_small_array_bytes(lv[l]);
  return s;
}

// Residual and restriction in one pass (a level's residual is read only by
// the restriction): C.b = P^T (b - A u), C.u = c C.b.  Two coarse columns a
// lane (fine columns f0 .. f0+3 of the lane and f0+4 of the next, as in
// mg_restrict); coarse rows march upwards, and the fine residual rows 2J,
// 2J+1, 2J+2 are formed in registers from a march over u, the even row shared
// between consecutive coarse rows.  The residual and the restriction take the
// operations of mg_stencil_pass and mg_restrict in the same order, so C.b is
// the same as from the two passes; the level's residual is never stored.
// write_u = 0: C.u (c C.b) is not stored; its first reader forms it from C.b.
template <class TM>
__global__ void __launch_bounds__(kGmThreads) k_gm_res_restrict(const GmScal* sc, MgLevel<TM> F, const TM* u,
                                                                MgLevel<TM> C, int write_u) {
  if (sc->stop) return;
  const Sched s = gm_sched(0);
  const Units un = make_units(C.nx, C.ny, 2, s.nw, 2);
  const Grid<const TM> gu{u, F.ld}, gb{F.b, F.ld};
  const Grid<TM> gcb{C.b, C.ld}, gcu{C.u, C.ld};
  const TM c = (TM)kMgC;
  for (int w = s.w; w < un.nunits; w += s.nw) {
    int st, y0, y1;
    unit_bounds(un, w, C.ny, st, y0, y1);
    const int xs = st * 128, f0 = xs + 4 * s.lane, I0 = f0 / 2;
    auto field = [&](int j, FRow<4, TM>& f) { field_plain<4>(gu, F.nx, F.ny, j, f0, xs, s.lane, f); };
    // residual of fine row j at columns f0 .. f0+4 (zero outside the grid)
    auto res_row = [&](int j, const FRow<4, TM>& S, const FRow<4, TM>& Cr, const FRow<4, TM>& N, TM (&r)[5]) {
      if (j < 0 || j >= F.ny) {
#pragma unroll
        for (int k = 0; k < 5; ++k) r[k] = TM(0);
        return;
      }
      TM ax[4], bv[4];
      stencil_row<4>(S, Cr, N, s.lane, ax);
      load_row<4>(gb, j, f0, F.nx, bv);
#pragma unroll
      for (int k = 0; k < 4; ++k) r[k] = f0 + k < F.nx ? bv[k] - ax[k] : TM(0);
      TM e = __shfl_down_sync(0xffffffffu, r[0], 1);
      if (s.lane == 31) {  // column xs + 128: the next strip's first, formed here
        const int xe = xs + 128;
        e = TM(0);
        if (xe < F.nx) {
          TM acc = TM(4) * Cr.hr;
          acc -= Cr.f[3];
          acc -= xe + 1 < F.nx ? gu.row(j)[xe + 1] : TM(0);
          acc -= S.hr;
          acc -= N.hr;
          e = gb.row(j)[xe] - acc;
        }
      }
      r[4] = e;
    };
    FRow<4, TM> fS, fC, fN;
    TM lo[5], mid[5], hi[5];
    int j = 2 * y0;
    field(j - 1, fS);
    field(j, fC);
    field(j + 1, fN);
    res_row(j, fS, fC, fN, lo);
    for (int J = y0; J < y1; ++J) {
      fS = fC; fC = fN; field(2 * J + 2, fN);
      res_row(2 * J + 1, fS, fC, fN, mid);
      fS = fC; fC = fN; field(2 * J + 3, fN);
      res_row(2 * J + 2, fS, fC, fN, hi);
      TM bc[2], uc[2];
#pragma unroll
      for (int q = 0; q < 2; ++q) {
        const int wq = 2 * q, m = wq + 1, e = wq + 2;
        const TM s1 = ((mid[wq] + mid[e]) + lo[m]) + hi[m];
        const TM s2 = ((lo[wq] + lo[e]) + hi[wq]) + hi[e];
        bc[q] = TM(0.25) * ((TM(4) * mid[m] + TM(2) * s1) + s2);
        uc[q] = c * bc[q];
      }
      store_row<2>(gcb, J, I0, C.nx, bc);
      if (write_u) store_row<2>(gcu, J, I0, C.nx, uc);
#pragma unroll
      for (int k = 0; k < 5; ++k) lo[k] = hi[k];
    }
  }
}

// A level's whole descent for nu = 2 in one pass (binary32 V-cycle): the
// second pre-smoothing sweep v = c b + c (b - A c b) (the first, c b, from
// zero), stored, and from v the residual b - A v restricted to the coarse
// level as in k_gm_res_restrict.  The march runs over b: v rows are formed one
// row ahead of the residual rows that need them (b two rows ahead).  The
// strip's halo columns of v (xs - 1; xs + 128 and xs + 129 for the residual
// at the next strip's first column) are formed point-wise by lanes 0 and 31.
// A unit stores the v rows of its coarse rows (fine rows 2 y0 .. 2 y1 - 1; the
// last unit also the rows above), the last strip also the columns past it.
// Same operations in the same order as the separate sweep and residual.
template <class TM>
__global__ void __launch_bounds__(kGmThreads) k_gm_jac_res_restrict(const GmScal* sc, MgLevel<TM> F, TM* vout,
                                                                    MgLevel<TM> C, int write_u) {
  if (sc->stop) return;
  const Sched s = gm_sched(0);
  const Units un = make_units(C.nx, C.ny, 2, s.nw, 2);
  const Grid<const TM> gb{F.b, F.ld};
  const Grid<TM> gv{vout, F.ld}, gcb{C.b, C.ld}, gcu{C.u, C.ld};
  const TM c = (TM)kMgC;
  const int lane = s.lane;
  auto cb_at = [&](int i, int x) -> TM {
    return (i < 0 || i >= F.ny || x < 0 || x >= F.nx) ? TM(0) : c * gb.row(i)[x];
  };
  auto v_at = [&](int i, int x) -> TM {  // the sweep at one point
    if (i < 0 || i >= F.ny || x < 0 || x >= F.nx) return TM(0);
    const TM cc = cb_at(i, x);
    TM acc = TM(4) * cc;
    acc -= cb_at(i, x - 1);
    acc -= cb_at(i, x + 1);
    acc -= cb_at(i - 1, x);
    acc -= cb_at(i + 1, x);
    return mg_fma(c, gb.row(i)[x] - acc, cc);
  };
  for (int w = s.w; w < un.nunits; w += s.nw) {
    int st, y0, y1;
    unit_bounds(un, w, C.ny, st, y0, y1);
    const int xs = st * 128, f0 = xs + 4 * lane, I0 = f0 / 2;
    const bool last_strip = (st == un.ns - 1), top = (y1 == C.ny);
    // b of row i (zero outside the grid) as loaded, then scaled to c b with b
    // itself kept for the lane's columns; the march loads a row one step
    // before it scales and uses it, so the load's latency overlaps a row's work
    auto b_load = [&](int i, FRow<4, TM>& f) { field_plain<4>(gb, F.nx, F.ny, i, f0, xs, lane, f); };
    auto cb_scale = [&](FRow<4, TM>& f, TM (&raw)[5]) {
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        raw[k] = f.f[k];
        f.f[k] = c * f.f[k];
      }
      raw[4] = f.hr;  // lane 31: b at column xs + 128, for the residual there
      f.hl = c * f.hl;
      f.hr = c * f.hr;
    };
    auto cb_row = [&](int i, FRow<4, TM>& f, TM (&raw)[5]) {
      b_load(i, f);
      cb_scale(f, raw);
    };
    // v of row i from c b rows i-1, i, i+1 (bv: b of row i); hr2: v at xs + 129 (lane 31)
    auto v_row = [&](int i, const FRow<4, TM>& S, const FRow<4, TM>& Cr, const TM (&bv)[5], const FRow<4, TM>& N,
                     FRow<4, TM>& v, TM& hr2) {
      if (i < 0 || i >= F.ny) {
        v.zero();
        hr2 = TM(0);
        return;
      }
      TM ax[4];
      stencil_row<4>(S, Cr, N, lane, ax);
#pragma unroll
      for (int k = 0; k < 4; ++k) v.f[k] = f0 + k < F.nx ? mg_fma(c, bv[k] - ax[k], Cr.f[k]) : TM(0);
      // the three halo points in one divergent branch: lane 0 forms column
      // xs - 1, lane 31 column xs + 128 and lane 30 column xs + 129, which
      // lane 31 then takes by a shuffle
      TM h = TM(0);
      if (lane == 0 || lane >= 30) h = v_at(i, lane == 0 ? xs - 1 : lane == 31 ? xs + 128 : xs + 129);
      const TM h30 = __shfl_up_sync(0xffffffffu, h, 1);
      v.hl = (lane == 0) ? h : TM(0);
      v.hr = (lane == 31) ? h : TM(0);
      hr2 = (lane == 31) ? h30 : TM(0);
    };
    auto store_v = [&](int i, const FRow<4, TM>& v, TM hr2) {
      if (i < 0 || i >= F.ny) return;
      store_row<4>(gv, i, f0, F.nx, v.f);
      if (last_strip && lane == 31) {  // columns past the last strip
        if (xs + 128 < F.nx) gv.row(i)[xs + 128] = v.hr;
        if (xs + 129 < F.nx) gv.row(i)[xs + 129] = hr2;
      }
    };
    // residual of row j at columns f0 .. f0+4 from v rows j-1, j, j+1 (bv: b of row j)
    auto res_row = [&](int j, const FRow<4, TM>& S, const FRow<4, TM>& Cr, TM crh2, const FRow<4, TM>& N,
                       const TM (&bv)[5], TM (&r)[5]) {
      if (j < 0 || j >= F.ny) {
#pragma unroll
        for (int k = 0; k < 5; ++k) r[k] = TM(0);
        return;
      }
      TM ax[4];
      stencil_row<4>(S, Cr, N, lane, ax);
#pragma unroll
      for (int k = 0; k < 4; ++k) r[k] = f0 + k < F.nx ? bv[k] - ax[k] : TM(0);
      TM e = __shfl_down_sync(0xffffffffu, r[0], 1);
      if (lane == 31) {
        const int xe = xs + 128;
        e = TM(0);
        if (xe < F.nx) {
          TM acc = TM(4) * Cr.hr;
          acc -= Cr.f[3];
          acc -= crh2;
          acc -= S.hr;
          acc -= N.hr;
          e = bv[4] - acc;
        }
      }
      r[4] = e;
    };
    // march state: c b rows (bA, bB, bC) = rows i-1, i, i+1 of the last v row i,
    // with b of the same rows (rA, rB, rC; element 4: column xs + 128); v rows (vS, vC, vN) with their hr2
    // for the next residual row (whose b row is then rA)
    FRow<4, TM> bA, bB, bC, bD, vS, vC, vN;  // bD: b of row i + 2, loaded ahead
    TM rA[5], rB[5], rC[5];
    TM hS, hC, hN;
    int i = 2 * y0 - 1;  // the last v row formed
    cb_row(i - 1, bA, rA);
    cb_row(i, bB, rB);
    cb_row(i + 1, bC, rC);
    b_load(i + 2, bD);
    v_row(i, bA, bB, rB, bC, vS, hS);
    auto next_v = [&](FRow<4, TM>& v, TM& h) {  // v row i + 1, advancing the b rows
      ++i;
      bA = bB;
      bB = bC;
      bC = bD;
#pragma unroll
      for (int k = 0; k < 5; ++k) {
        rA[k] = rB[k];
        rB[k] = rC[k];
      }
      cb_scale(bC, rC);
      b_load(i + 2, bD);
      v_row(i, bA, bB, rB, bC, v, h);
    };
    next_v(vC, hC);  // row 2 y0
    next_v(vN, hN);  // row 2 y0 + 1
    store_v(2 * y0, vC, hC);
    TM lo[5], mid[5], hi[5];
    res_row(2 * y0, vS, vC, hC, vN, rA, lo);
    for (int J = y0; J < y1; ++J) {
      vS = vC; vC = vN; hC = hN;
      next_v(vN, hN);  // row 2J + 2
      res_row(2 * J + 1, vS, vC, hC, vN, rA, mid);
      store_v(2 * J + 1, vC, hC);
      vS = vC; vC = vN; hC = hN;
      next_v(vN, hN);  // row 2J + 3
      res_row(2 * J + 2, vS, vC, hC, vN, rA, hi);
      if (J + 1 < y1 || top) store_v(2 * J + 2, vC, hC);
      TM bcv[2], ucv[2];
#pragma unroll
      for (int q = 0; q < 2; ++q) {
        const int wq = 2 * q, m = wq + 1, e = wq + 2;
        const TM s1 = ((mid[wq] + mid[e]) + lo[m]) + hi[m];
        const TM s2 = ((lo[wq] + lo[e]) + hi[wq]) + hi[e];
        bcv[q] = TM(0.25) * ((TM(4) * mid[m] + TM(2) * s1) + s2);
        ucv[q] = c * bcv[q];
      }
      store_row<2>(gcb, J, I0, C.nx, bcv);
      if (write_u) store_row<2>(gcu, J, I0, C.nx, ucv);
#pragma unroll
      for (int k = 0; k < 5; ++k) lo[k] = hi[k];
    }
    if (top) store_v(2 * y1 + 1, vN, hN);  // the grid's last fine row, above the last coarse row's
  }
}

// Prolongation and the first post-smoothing sweep in one pass: out = u' + c (b -
// A u') with u' = u + P e, u' formed in registers (never stored).  Tiles as in
// k_gm_sweep, with one group of four columns a lane (the prolongation's lane
// layout); the coarse values a lane needs (3 coarse rows x 3 columns, 4 for
// lane 31's halo) are read once per tile.  u' takes mg_prolong's operations
// and the sweep mg_stencil_pass's, in the same order.
template <class TM>
__global__ void __launch_bounds__(kGmThreads) k_gm_prolong_jac(const GmScal* sc, MgLevel<TM> L, const TM* u,
                                                               MgLevel<TM> C, const TM* e, TM* out) {
  if (sc->stop) return;
  constexpr int V = 4, R = 2;
  static_assert(R == 2, "cv holds the three coarse rows of R + 2 = 4 fine rows");
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, wpc = blockDim.x >> 5;
  const int ns = (L.nx + 32 * V - 1) / (32 * V);
  const int band = wpc * R;
  const int ntiles = ns * ((L.ny + band - 1) / band);
  const Grid<const TM> gu{u, L.ld}, gb{L.b, L.ld}, ge{e, C.ld};
  const Grid<TM> go{out, L.ld};
  const TM c = (TM)kMgC;
  auto ce = [&](int I, int J) -> TM { return (I < 0 || I >= C.nx || J < 0 || J >= C.ny) ? TM(0) : ge.row(J)[I]; };
  for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
    const int st = t % ns;
    const int jb = (t / ns) * band + warp * R;  // even
    if (jb >= L.ny) continue;
    const int xs = st * 32 * V, f0 = xs + 4 * lane, I0 = f0 / 2, Jc0 = jb / 2 - 1;
    // coarse rows Jc0 .. Jc0+2, columns I0-1 .. I0+2 (the last for lane 31's halo)
    TM cv[3][4];
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
      for (int q = 0; q < 4; ++q) cv[a][q] = (q == 3 && lane != 31) ? TM(0) : ce(I0 - 1 + q, Jc0 + a);
    // u' of fine row j = jb - 1 + k: the lane's 4 columns, and the strip's halo
    // columns (jb is even: k = 0, 2 are odd rows on coarse row k / 2 of cv,
    // k = 1, 3 even rows between coarse rows (k - 1) / 2 and (k + 1) / 2)
    auto field = [&](int k, FRow<V, TM>& f) {
      const int j = jb - 1 + k;
      if (j < 0 || j >= L.ny) { f.zero(); return; }
      field_plain<V>(gu, L.nx, L.ny, j, f0, xs, lane, f);
      TM v[4], vl, vr;
      if ((k & 1) == 0) {
        const int a = k >> 1;
        v[0] = TM(0.5) * (cv[a][0] + cv[a][1]);
        v[1] = cv[a][1];
        v[2] = TM(0.5) * (cv[a][1] + cv[a][2]);
        v[3] = cv[a][2];
        vl = cv[a][0];                                  // column f0 - 1 (odd): coarse I0 - 1
        vr = TM(0.5) * (cv[a][2] + cv[a][3]);           // column f0 + 4 (even)
      } else {
        const int ia = (k + 1) >> 1, ib = ia - 1;
        v[0] = TM(0.25) * ((cv[ib][0] + cv[ib][1]) + (cv[ia][0] + cv[ia][1]));
        v[1] = TM(0.5) * (cv[ib][1] + cv[ia][1]);
        v[2] = TM(0.25) * ((cv[ib][1] + cv[ib][2]) + (cv[ia][1] + cv[ia][2]));
        v[3] = TM(0.5) * (cv[ib][2] + cv[ia][2]);
        vl = TM(0.5) * (cv[ib][0] + cv[ia][0]);
        vr = TM(0.25) * ((cv[ib][2] + cv[ib][3]) + (cv[ia][2] + cv[ia][3]));
      }
#pragma unroll
      for (int k = 0; k < 4; ++k) f.f[k] = f0 + k < L.nx ? f.f[k] + v[k] : TM(0);
      if (lane == 0) f.hl = (xs >= 1 && xs - 1 < L.nx) ? f.hl + vl : TM(0);
      if (lane == 31) f.hr = (xs + 32 * V < L.nx) ? f.hr + vr : TM(0);
    };
    FRow<V, TM> fr[R + 2];
#pragma unroll
    for (int k = 0; k < R + 2; ++k) field(k, fr[k]);
#pragma unroll
    for (int k = 0; k < R; ++k) {
      const int j = jb + k;
      if (j >= L.ny) break;
      TM ax[V], bv[V], o[V];
      load_row<V>(gb, j, f0, L.nx, bv);
      stencil_row<V>(fr[k], fr[k + 1], fr[k + 2], lane, ax);
#pragma unroll
      for (int q = 0; q < V; ++q) o[q] = mg_fma(c, bv[q] - ax[q], fr[k + 1].f[q]);
      store_row<V>(go, j, f0, L.nx, o);
    }
  }
}

// The levels [first, nlev) on the calling CTA (every thread of it), resident
// in its dynamic shared memory when SMEM (else in global memory); level
// `first`'s final iterate ends in its global buffer (u or v as the V-cycle's
// parity says).  lv: a shared-memory array of kMgMaxLevels descriptors.
template <class TM, bool SMEM>
__device__ void gm_small_levels(const GmLevels<TM>& levels, int nlev, int first, int nu, int nu_c,
                                unsigned char* gsm, MgLevel<TM>* lv) {
  if (threadIdx.x == 0) {
    size_t off = 0;
    for (int l = 0; l < kMgMaxLevels; ++l) {
      MgLevel<TM> L = levels.lv[l];
      if (SMEM && l >= first && l < nlev) {
        const size_t nb = gm_small_array_bytes(L);
        L.b = reinterpret_cast<TM*>(gsm + off);
        L.u = reinterpret_cast<TM*>(gsm + off + nb);
        L.v = reinterpret_cast<TM*>(gsm + off + 2 * nb);
        off += 3 * nb;
      }
      lv[l] = L;
    }
  }
  __syncthreads();
  // level `first`'s first sweep from zero, c b, formed here (its producer may
  // not have stored it)
  const MgLevel<TM>& G = levels.lv[first];
  const int n0 = G.ny * G.ld;
  const TM c = (TM)kMgC;
  for (int i0 = threadIdx.x; i0 < n0; i0 += 4 * blockDim.x) {  // four loads in flight a thread
    TM bi[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const int i = i0 + k * (int)blockDim.x;
      bi[k] = i < n0 ? G.b[i] : TM(0);
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const int i = i0 + k * (int)blockDim.x;
      if (i < n0) {
        if (SMEM) lv[first].b[i] = bi[k];
        lv[first].u[i] = c * bi[k];
      }
    }
  }
  __syncthreads();
  const int par = tiny_vcycle<TM>(lv, nlev, first, nu, nu_c);
  if (SMEM) {
    const TM* res = par ? lv[first].v : lv[first].u;
    TM* dst = par ? G.v : G.u;
    for (int i = threadIdx.x; i < n0; i += blockDim.x) dst[i] = res[i];
  }
}

// Which buffer holds level l's iterate after a V-cycle from l: 2 nu - 1 sweeps
// (nu - 1 down, nu up), or nu_c - 1 on the coarsest level.
__host__ __device__ inline int gm_final_parity(int l, int nlev, int nu, int nu_c) {
  return (l < nlev - 1 ? 2 * nu - 1 : nu_c - 1) & 1;
}

// SMEM = false: the levels stay in global memory (shapes whose levels do not
// fit in shared memory, e.g. one column wide with a padded pitch).
template <class TM, bool SMEM>
__global__ void __launch_bounds__(512) k_gm_small(const GmScal* sc, GmLevels<TM> levels, int nlev, int first, int nu,
                                                  int nu_c) {
  if (sc->stop) return;
  extern __shared__ __align__(16) unsigned char gsm[];
  __shared__ MgLevel<TM> lv[kMgMaxLevels];
  gm_small_levels<TM, SMEM>(levels, nlev, first, nu, nu_c, gsm, lv);
}

// r = b - A x, level 0: b = r (rounded to TM), u = c b (write_u); partials
// (b, b), (r, r).
template <class TM>
__global__ void __launch_bounds__(kGmThreads) k_gm_init(const GmBind* bd, double* part, int nx, int ny, int ld,
                                                         Grid<double> r, MgLevel<TM> L0, int write_u) {
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
      // x = 0 on these three rows (the usual zero start): A x = 0 without the
      // binary64 stencil, whose 4 operations a point on the FP64 pipe are most
      // of this pass (a warp-uniform test on the bits)
      bool zero = ((__double_as_longlong(C.hl) | __double_as_longlong(C.hr)) << 1) == 0;
#pragma unroll
      for (int k = 0; k < V; ++k)
        zero = zero && ((__double_as_longlong(S.f[k]) | __double_as_longlong(C.f[k]) |
                         __double_as_longlong(N.f[k])) << 1) == 0;
      if (__all_sync(0xffffffffu, zero)) {
#pragma unroll
        for (int k = 0; k < V; ++k) ax[k] = 0.0;
      } else {
        stencil_row<V>(S, C, N, s.lane, ax);
      }
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
      if (write_u) store_row<V>(g0u, j, xl, nx, ru);
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

// p = z + beta p (halo included), q = A p, partial (p, q); and the previous
// iteration's x += alpha p with that p (read here anyway), deferred from the
// x, r pass (which then moves 16 bytes a point fewer).
template <class TM>
__global__ void __launch_bounds__(kGmThreads) k_gm_pq(const GmScal* sc, const GmBind* bd, double* part, int nx,
                                                       int ny, int ld, Grid<double> p0, Grid<double> p1,
                                                       Grid<double> q, MgLevel<TM> L0, int zbuf, int rev) {
  if (sc->stop) return;
  constexpr int V = 2;
  const Sched s = gm_sched(rev);
  const Units un = make_units(nx, ny, V, s.nw, 2);
  const double beta = sc->beta;
  const bool first = (sc->iters == 0);
  const bool xp = sc->xpend != 0;
  const double alpha_old = sc->alpha;
  const Grid<double> x{bd->x, ld};
  const Grid<double> pold = sc->cur ? p1 : p0;
  const Grid<double> pnew = sc->cur ? p0 : p1;
  const Grid<const TM> gz{zbuf ? L0.v : L0.u, L0.ld};
  Acc64 apq;
  struct D { double x[V], p[V]; };
  for (int u = s.w; u < un.nunits; u += s.nw) {
    int st, y0, y1;
    unit_bounds(un, u, ny, st, y0, y1);
    const int xs = st * 32 * V, xl = Lanes<V>::first(xs, s.lane);
    const int nval = nx - xl;
    auto zone = [&](int j, int xx) -> double { return (xx < 0 || xx >= nx) ? 0.0 : mg_widen(gz.row(j)[xx]); };
    auto pone = [&](int j, int xx) -> double { return (xx < 0 || xx >= nx) ? 0.0 : pold.row(j)[xx]; };
    auto field = [&](int j, FRow<V, double>& f) {
      if (j < 0 || j >= ny) { f.zero(); return; }
      TM zt[V];
      load_row<V>(gz, j, xl, nx, zt);
      if (first) {
#pragma unroll
        for (int k = 0; k < V; ++k) f.f[k] = mg_widen(zt[k]);
        f.hl = (s.lane == 0) ? zone(j, xs - 1) : 0.0;
        f.hr = (s.lane == 31) ? zone(j, xs + 32 * V) : 0.0;
      } else {
        double pv[V];
        load_row<V>(pold, j, xl, nx, pv);
#pragma unroll
        for (int k = 0; k < V; ++k) f.f[k] = __fma_rn(beta, pv[k], mg_widen(zt[k]));
        f.hl = (s.lane == 0) ? __fma_rn(beta, pone(j, xs - 1), zone(j, xs - 1)) : 0.0;
        f.hr = (s.lane == 31) ? __fma_rn(beta, pone(j, xs + 32 * V), zone(j, xs + 32 * V)) : 0.0;
      }
    };
    auto load = [&](int j, D& d) {
      if (xp) {
        load_row<V>(x, j, xl, nx, d.x);
        load_row<V>(pold, j, xl, nx, d.p);
      }
    };
    auto finish = [&](int j, const D& d, const FRow<V, double>& S, const FRow<V, double>& C,
                      const FRow<V, double>& N) {
      double qv[V];
      stencil_row<V>(S, C, N, s.lane, qv);
      store_row<V>(pnew, j, xl, nx, C.f);
      store_row<V>(q, j, xl, nx, qv);
      acc_dot<V>(apq, j, C.f, qv, nval);
      if (xp) {
        double xv[V];
#pragma unroll
        for (int k = 0; k < V; ++k) xv[k] = __fma_rn(alpha_old, d.p[k], d.x[k]);
        store_row<V>(x, j, xl, nx, xv);
      }
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
  sc->xpend = 0;  // k_gm_pq applied the previous x update
  if (!(pq > 0.0) || !isfinite(pq)) {
    sc->status = LAP5CG_ERR_BREAKDOWN;
    sc->stop = 1;
    return;
  }
  sc->alpha = sc->gamma / pq;
  sc->cur ^= 1;
}

// r -= alpha q, partial (r, r); level 0: b = r, u = c b (write_u).  (x += alpha p
// is left to the next p, q pass or, after the loop, to k_gm_xfinal.)
template <class TM>
__global__ void __launch_bounds__(kGmThreads) k_gm_xr(const GmScal* sc, double* part, int nx, int ny,
                                                       Grid<double> r, Grid<double> q, MgLevel<TM> L0, int rev,
                                                       int write_u) {
  if (sc->stop) return;
  constexpr int V = 2;
  const Sched s = gm_sched(rev);
  const Units un = make_units(nx, ny, V, s.nw, 2);
  const double alpha = sc->alpha;
  const Grid<TM> g0b{L0.b, L0.ld}, g0u{L0.u, L0.ld};
  const TM cm = (TM)kMgC;
  Acc64 arr;
  struct D { double r[V], q[V]; };
  for (int u = s.w; u < un.nunits; u += s.nw) {
    int st, y0, y1;
    unit_bounds(un, u, ny, st, y0, y1);
    const int xl = Lanes<V>::first(st * 32 * V, s.lane);
    const int nval = nx - xl;
    auto load = [&](int j, D& d) {
      load_row<V>(r, j, xl, nx, d.r);
      load_row<V>(q, j, xl, nx, d.q);
    };
    auto finish = [&](int j, const D& d) {
      double rv[V];
      TM rb[V], ru[V];
#pragma unroll
      for (int k = 0; k < V; ++k) {
        rv[k] = __fma_rn(-alpha, d.q[k], d.r[k]);
        rb[k] = (TM)rv[k];
        ru[k] = cm * rb[k];
      }
      acc_dot<V>(arr, j, rv, rv, nval);
      store_row<V>(r, j, xl, nx, rv);
      store_row<V>(g0b, j, xl, nx, rb);
      if (write_u) store_row<V>(g0u, j, xl, nx, ru);
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
  s.xpend = 1;  // this iteration's x += alpha p is pending
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

// After the loop: the pending x += alpha p (the last x, r pass's).
__global__ void __launch_bounds__(kGmThreads) k_gm_xfinal(const GmScal* sc, const GmBind* bd, int nx, int ny, int ld,
                                                           Grid<double> p0, Grid<double> p1) {
  if (!sc->xpend) return;
  const double alpha = sc->alpha;
  const Grid<double> p = sc->cur ? p1 : p0;
  double* x = bd->x;
  const long long n = (long long)nx * ny;
  for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x) {
    const int j = (int)(t / nx), i = (int)(t - (long long)j * nx);
    x[(size_t)j * ld + i] = __fma_rn(alpha, p.row(j)[i], x[(size_t)j * ld + i]);
  }
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
  const TM* e;     // GP_PROLONG_JAC: the coarse iterate
  int from_b = 0;  // GP_JAC: the input iterate is c b, formed from the level's b
};

// The V-cycle's passes on the big levels as Vcycle::run executes them (buffer
// parities and march directions), with the single-CTA levels as one entry
// (kind -1).  fuse (binary32 V-cycle): residual + restriction and
// prolongation + first post-smoothing sweep are single passes, and where every
// level's first reader of its first sweep c b is a Jacobi sweep (*write_u =
// false), that sweep forms c b from b and no producer stores it.  (A binary64
// V-cycle keeps the separate passes: its fused forms measured slower, the
// arithmetic, not the traffic, being its limit.)  Returns the buffer that
// holds level 0's result (M^-1 r).
template <class TM>
static int gm_pass_list(const PcgArgs<TM>& a, bool fuse, std::vector<GmPassRec<TM>>& out, bool* write_u) {
  const int L = a.nlev, nu = a.nu;
  *write_u = !fuse || nu < 2 || (a.lsmall >= L && a.nu_c < 2);
  const int fb = *write_u ? 0 : 1;
  int cur[kMgMaxLevels] = {0};
  unsigned pc = 0;
  auto it = [&](int l) -> TM* { return cur[l] ? a.lv[l].v : a.lv[l].u; };
  auto other = [&](int l) -> TM* { return cur[l] ? a.lv[l].u : a.lv[l].v; };
  auto jac = [&](int l, bool last, int from_b) {
    out.push_back({last ? GP_JAC_DOT : GP_JAC, l, (int)(pc++ & 1u), it(l), other(l), nullptr, from_b});
    cur[l] ^= 1;
  };
  auto sweeps = [&](int l, int n, bool final0) {  // sweeps 2 .. n (the first, c b, came with b)
    for (int k = 1; k < n; ++k) jac(l, final0 && l == 0 && k == n - 1, k == 1 ? fb : 0);
  };
  const int big_end = a.lsmall < L - 1 ? a.lsmall : L - 1;
  for (int l = 0; l < big_end; ++l) {  // down: pre-smoothing, residual, restriction
    if (fuse && nu == 2) {  // the one explicit sweep, residual and restriction: one pass
      out.push_back({GP_JAC_RES_RESTRICT, l, (int)(pc++ & 1u), nullptr, other(l), nullptr});
      cur[l] ^= 1;
      cur[l + 1] = 0;
      continue;
    }
    sweeps(l, nu, false);
    if (fuse) {
      out.push_back({GP_RES_RESTRICT, l, (int)(pc++ & 1u), it(l), nullptr, nullptr});
    } else {
      out.push_back({GP_RES, l, (int)(pc++ & 1u), it(l), other(l), nullptr});
      out.push_back({GP_RESTRICT, l, (int)(pc++ & 1u), other(l), nullptr, nullptr});
    }
    cur[l + 1] = 0;
  }
  if (a.lsmall >= L) {
    sweeps(L - 1, a.nu_c, false);
  } else {
    out.push_back({-1, big_end, 0, nullptr, nullptr, nullptr});
    cur[big_end] = gm_final_parity(big_end, L, nu, a.nu_c);
  }
  for (int l = big_end - 1; l >= 0; --l) {  // up: prolongation, post-smoothing
    int k0 = 0;
    if (fuse && !(l == 0 && nu == 1)) {  // (level 0's only sweep is the (r, z) sweep: not fused)
      out.push_back({GP_PROLONG_JAC, l, (int)(pc++ & 1u), it(l), other(l), it(l + 1)});
      cur[l] ^= 1;
      k0 = 1;
    } else {
      out.push_back({GP_PROLONG, l, (int)(pc++ & 1u), it(l + 1), it(l), nullptr});
    }
    for (int k = k0; k < nu; ++k) jac(l, l == 0 && k == nu - 1, 0);
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

static int gm_add(cudaGraph_t g, cudaGraphNode_t* prev, const void* fn, unsigned grid, unsigned block, void** args,
                  unsigned smem = 0) {
  cudaKernelNodeParams kp = {};
  kp.func = const_cast<void*>(fn);
  kp.gridDim = dim3(grid);
  kp.blockDim = dim3(block);
  kp.sharedMemBytes = smem;
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
  const void* f_sweep_j = reinterpret_cast<const void*>(&k_gm_sweep<TM, GP_JAC>);
  const void* f_sweep_r = reinterpret_cast<const void*>(&k_gm_sweep<TM, GP_RES>);
  // (c b formed from b: binary32 V-cycles only)
  const void* f_sweep_jb = reinterpret_cast<const void*>(&k_gm_sweep<TM, GP_JAC, sizeof(TM) == 4>);
  const void* f_sweep_d = reinterpret_cast<const void*>(&k_gm_sweep<TM, GP_JAC_DOT>);
  const int nb_dot_max = gm_blocks(f_sweep_d, kGmThreads, dp.sms);
  int nb_dot = nb_pass;  // CTAs of the (r, z) sweep
  const int nb_sweep = gm_blocks(f_sweep_j, kGmThreads, dp.sms);
  const void* f_rr = reinterpret_cast<const void*>(&k_gm_res_restrict<TM>);
  const void* f_pj = reinterpret_cast<const void*>(&k_gm_prolong_jac<TM>);
  const int nb_rr = gm_blocks(f_rr, kGmThreads, dp.sms);
  const void* f_jrr = reinterpret_cast<const void*>(&k_gm_jac_res_restrict<TM>);
  const int nb_jrr = gm_blocks(f_jrr, kGmThreads, dp.sms);
  const int nb_pj = gm_blocks(f_pj, kGmThreads, dp.sms);
  const int nb_init = gm_blocks(f_init, kGmThreads, dp.sms);
  const int nb_pq = gm_blocks(f_pq, kGmThreads, dp.sms);
  const int nb_xr = gm_blocks(f_xr, kGmThreads, dp.sms);
  const int nb_true = gm_blocks(f_true, kGmThreads, dp.sms);
  std::vector<GmPassRec<TM>> passes;
  bool wu = true;
  const int zbuf = gm_pass_list<TM>(a, sizeof(TM) == 4, passes, &wu);
  int write_u = wu ? 1 : 0;

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
    void* args[] = {&bd, &part, &nx_, &ny_, &ld_, &gr, &L0, &write_u};
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
        // the levels in shared memory where they fit
        size_t smem = gm_small_smem<TM>(a.lv, first, nlev);
        const void* fs = reinterpret_cast<const void*>(&k_gm_small<TM, true>);
        cudaFuncAttributes fa;
        if (cudaFuncGetAttributes(&fa, fs) != cudaSuccess) return fail(LAP5CG_ERR_CUDA);
        if (smem + fa.sharedSizeBytes <= (size_t)dp.max_smem_optin) {
          if (cudaFuncSetAttribute(fs, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
            return fail(LAP5CG_ERR_CUDA);
        } else {
          fs = reinterpret_cast<const void*>(&k_gm_small<TM, false>);
          smem = 0;
        }
        if ((rc = gm_add(body, &bp, fs, 1, 512, args, (unsigned)smem)) != LAP5CG_OK) return fail(rc);
        continue;
      }
      MgLevel<TM> L = a.lv[pr.level];
      MgLevel<TM> Lc = a.lv[pr.level + 1 < a.nlev ? pr.level + 1 : pr.level];
      int kind = pr.kind, rev = pr.rev;
      const TM* in = pr.in;
      TM* out = pr.out;
      const int wpc = kGmThreads / 32;
      if (kind == GP_JAC_RES_RESTRICT) {
        const Units un = make_units(Lc.nx, Lc.ny, 2, 1ll << 40, 2);
        const int grid = (int)std::min<long long>(((long long)un.nunits + wpc - 1) / wpc, nb_jrr);
        void* jargs[] = {&sc, &L, &out, &Lc, &write_u};
        if ((rc = gm_add(body, &bp, f_jrr, (unsigned)(grid < 1 ? 1 : grid), kGmThreads, jargs)) != LAP5CG_OK)
          return fail(rc);
        continue;
      }
      if (kind == GP_RES_RESTRICT) {
        const Units un = make_units(Lc.nx, Lc.ny, 2, 1ll << 40, 2);
        const int grid = (int)std::min<long long>(((long long)un.nunits + wpc - 1) / wpc, nb_rr);
        const TM* uin = in;
        void* rargs[] = {&sc, &L, &uin, &Lc, &write_u};
        if ((rc = gm_add(body, &bp, f_rr, (unsigned)(grid < 1 ? 1 : grid), kGmThreads, rargs)) != LAP5CG_OK)
          return fail(rc);
        continue;
      }
      if (kind == GP_PROLONG_JAC) {
        const long long ntiles = (long long)((L.nx + 127) / 128) * ((L.ny + 2 * wpc - 1) / (2 * wpc));
        const int grid = (int)std::min<long long>(ntiles, nb_pj);
        const TM* uin = in;
        const TM* ein = pr.e;
        void* pargs[] = {&sc, &L, &uin, &Lc, &ein, &out};
        if ((rc = gm_add(body, &bp, f_pj, (unsigned)grid, kGmThreads, pargs)) != LAP5CG_OK) return fail(rc);
        continue;
      }
      if (kind == GP_JAC_DOT) {
        const int V = GmDotVec<TM>::V;
        const long long ntiles = (long long)((L.nx + 32 * V - 1) / (32 * V)) * ((L.ny + 2 * wpc - 1) / (2 * wpc));
        const int grid = (int)std::min<long long>(ntiles, nb_dot_max);
        nb_dot = grid;  // the partial sums k_gm_rz adds
        void* sargs[] = {&sc, &part, &L, &in, &out, &grc};
        if ((rc = gm_add(body, &bp, f_sweep_d, (unsigned)grid, kGmThreads, sargs)) != LAP5CG_OK) return fail(rc);
        continue;
      }
      if (kind == GP_JAC || kind == GP_RES) {
        // sweeps and residuals: the tiled kernel, as many CTAs as tiles up to
        // the resident maximum (binary32: two groups of four columns a lane;
        // the (r, z) sweep above keeps one, since its binary64 r rows in the
        // two-group layout took 104 registers and ran slower)
        const int V = GmSweepVec<TM>::V;
        const long long ntiles = (long long)((L.nx + 32 * V - 1) / (32 * V)) * ((L.ny + 2 * wpc - 1) / (2 * wpc));
        const void* fk = kind == GP_RES ? f_sweep_r : pr.from_b ? f_sweep_jb : f_sweep_j;
        const int grid = (int)std::min<long long>(ntiles, nb_sweep);
        void* sargs[] = {&sc, &part, &L, &in, &out, &grc};
        if ((rc = gm_add(body, &bp, fk, (unsigned)grid, kGmThreads, sargs)) != LAP5CG_OK) return fail(rc);
        continue;
      }
      // restriction and prolongation (the binary64 V-cycle's separate passes):
      // as many CTAs as the pass has warp units (two-row units), up to the
      // resident maximum -- the small levels' passes launch a few CTAs, not a
      // full grid of idle ones
      void* args[] = {&sc, &L, &Lc, &kind, &rev, &in, &out};
      int grid = nb_pass;
      {
        const long long kAll = 1ll << 40;
        const Units un = kind == GP_RESTRICT ? make_units(Lc.nx, Lc.ny, 2, kAll, 2) : make_units(L.nx, L.ny, 4, kAll, 2);
        const long long need = ((long long)un.nunits + wpc - 1) / wpc;
        if (need < grid) grid = need < 1 ? 1 : (int)need;
      }
      if ((rc = gm_add(body, &bp, f_pass, (unsigned)grid, kGmThreads, args)) != LAP5CG_OK) return fail(rc);
    }
    int nbp = nb_dot;
    {
      void* args[] = {&sc, &part, &nbp};
      if ((rc = gm_add(body, &bp, reinterpret_cast<const void*>(&k_gm_rz), 1, 256, args)) != LAP5CG_OK)
        return fail(rc);
    }
    int zb = zbuf, rev1 = 1, rev0 = 0;
    {
      void* args[] = {&sc, &bd, &part, &nx_, &ny_, &ld_, &gp0, &gp1, &gq, &L0, &zb, &rev1};
      if ((rc = gm_add(body, &bp, f_pq, nb_pq, kGmThreads, args)) != LAP5CG_OK) return fail(rc);
    }
    int nbq = nb_pq;
    {
      void* args[] = {&sc, &part, &nbq};
      if ((rc = gm_add(body, &bp, reinterpret_cast<const void*>(&k_gm_alpha), 1, 256, args)) != LAP5CG_OK)
        return fail(rc);
    }
    {
      void* args[] = {&sc, &part, &nx_, &ny_, &gr, &gq, &L0, &rev0, &write_u};
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
  {
    const void* f_xf = reinterpret_cast<const void*>(&k_gm_xfinal);
    void* args[] = {&sc, &bd, &nx_, &ny_, &ld_, &gp0, &gp1};
    if ((rc = gm_add(g, &prev, f_xf, gm_blocks(f_xf, kGmThreads, dp.sms), kGmThreads, args)) != LAP5CG_OK)
      return fail(rc);
  }
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
// takes the persistent kernel (the fine grid itself is a single-CTA level, the
// stream is capturing, or the graph cannot be built).
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
    if (rc != LAP5CG_OK) {  // a driver without conditional graph nodes: the persistent kernel solves
      cudaGetLastError();
      return LAP5CG_OK;
    }
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

// Every cached graph destroyed on its own device; the caller's current device
// is restored.
static int gm_release_all() {
  std::lock_guard<std::mutex> lock(g_gm_mu);
  int rc = LAP5CG_OK, dev0 = 0;
  const bool have_dev = cudaGetDevice(&dev0) == cudaSuccess;
  for (const auto& e : g_gm_cache) {
    if (cudaSetDevice(e.first.dev) != cudaSuccess || cudaGraphExecDestroy(e.second) != cudaSuccess)
      rc = LAP5CG_ERR_CUDA;
  }
  g_gm_cache.clear();
  if (have_dev) cudaSetDevice(dev0);
  if (rc != LAP5CG_OK) cudaGetLastError();
  return rc;
}

}  // namespace lap5

extern "C" LAP5CG_API int lap5cg_release_graphs(void) { return lap5::gm_release_all(); }
