// mg_kernels.cuh -- the multigrid V-cycle's device code (level layout, the
// Jacobi / residual, restriction and prolongation passes, and the V-cycle
// driver of the persistent kernels), shared by the persistent multigrid
// solves (mg.cu) and the graph-driven multigrid-preconditioned CG
// (mg_graph.cu).  See mg.cu for the method.
#pragma once

#include "cg_launch.cuh"

namespace lap5 {

constexpr int kMgMaxLevels = 24;
constexpr int kMgCtaPoints = 4096;  // levels this small run on one CTA
constexpr double kMgC = 0.2;         // omega / 4 with omega = 4/5

template <class TM>
struct MgLevel {
  int nx, ny, ld;  // ld a multiple of 4, rows 16-byte aligned
  TM *b, *u, *v;   // right-hand side and two iterate buffers
};

template <class TM>
struct PcgArgs {
  SolveCommon c;
  Grid<const double> b;
  Grid<double> x, r, p0, p1, q;  // p double-buffered: its halo is read while it is rewritten
  Grid<double> u, w, z, s;       // pipelined form: u = M^-1 r, w = A u, z, s (q and p0 as p shared)
  MgLevel<TM> lv[kMgMaxLevels];
  int nlev;    // levels (>= 1); level nlev-1 is the coarsest
  int lsmall;  // first level run by CTA 0 alone (nlev: none)
  int nu, nu_c;
};

// The warps taking part in a pass (all of the grid's, or CTA 0's) and the
// march direction (alternating from pass to pass keeps rows in L2).
struct Sched {
  int w, nw, lane;
  bool rev;
};

template <class TM> struct MgVec { static constexpr int V = 16 / (int)sizeof(TM); };  // one 16-byte vector a lane

__device__ __forceinline__ float mg_fma(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double mg_fma(double a, double b, double c) { return __fma_rn(a, b, c); }

// binary32 -> binary64 widening (exact) from the IEEE 754 formats: for a
// normal number the sign moves to bit 63, the exponent is re-biased by
// 1023 - 127 and the 23 fraction bits move up by 29; zeros keep their sign.
// Integer operations only: on GB300 the FP64 pipe (2 operations an SM a clock)
// is the limit of the binary64 PCG passes, and a hardware conversion would
// take a slot of it.  Subnormal, infinite and NaN inputs take the hardware
// conversion.
__device__ __forceinline__ double mg_widen(float f) {
  const uint32_t u = __float_as_uint(f);
  const uint32_t e = (u >> 23) & 0xffu;
  const unsigned long long s = (unsigned long long)(u >> 31) << 63;
  if (e - 1u < 254u)
    return __longlong_as_double(
        (long long)(s | ((unsigned long long)(e + 896u) << 52) | ((unsigned long long)(u & 0x7fffffu) << 29)));
  if ((u << 1) == 0u) return __longlong_as_double((long long)s);
  return (double)f;
}
__device__ __forceinline__ double mg_widen(double d) { return d; }

// Damped Jacobi sweep (JAC) out = in + c (b - A in), or residual out = b - A in;
// with DOT also accumulates (r, out) against the binary64 grid r (level 0).
template <class TM, bool JAC, bool DOT>
__device__ void mg_stencil_pass(const Sched& s, const MgLevel<TM>& L, const TM* in, TM* out,
                                const Grid<const double>& r, Acc64& acc) {
  constexpr int V = MgVec<TM>::V;
  const Units un = make_units(L.nx, L.ny, V, s.nw, 2);
  const Grid<const TM> gi{in, L.ld}, gb{L.b, L.ld};
  const Grid<TM> go{out, L.ld};
  const TM c = (TM)kMgC;
  struct D { TM b[V]; };
  for (int u = s.w; u < un.nunits; u += s.nw) {
    int st, y0, y1;
    unit_bounds(un, u, L.ny, st, y0, y1);
    const int xs = st * 32 * V, xl = Lanes<V>::first(xs, s.lane);
    const int nval = L.nx - xl;
    auto field = [&](int j, FRow<V, TM>& f) { field_plain<V>(gi, L.nx, L.ny, j, xl, xs, s.lane, f); };
    auto load = [&](int j, D& d) { load_row<V>(gb, j, xl, L.nx, d.b); };
    auto finish = [&](int j, const D& d, const FRow<V, TM>& S, const FRow<V, TM>& C, const FRow<V, TM>& N) {
      TM ax[V], o[V];
      stencil_row<V>(S, C, N, s.lane, ax);
#pragma unroll
      for (int k = 0; k < V; ++k) o[k] = JAC ? mg_fma(c, d.b[k] - ax[k], C.f[k]) : d.b[k] - ax[k];
      store_row<V>(go, j, xl, L.nx, o);
      if constexpr (DOT) {
        double rv[V], zv[V];
        load_row<V>(r, j, xl, L.nx, rv);
#pragma unroll
        for (int k = 0; k < V; ++k) zv[k] = mg_widen(o[k]);
        acc_dot<V>(acc, j, rv, zv, nval);
      }
    };
    march<V, TM, D>(y0, y1, s.rev, field, load, finish);
  }
}

// Fine values 2I0 .. 2I0+4 of row j for a lane whose coarse columns are I0,
// I0+1 (2I0 a multiple of 4): one vector load, the fifth from the next lane.
template <class TM>
__device__ __forceinline__ void mg_fine5(const Grid<const TM>& g, int nx, int ny, int j, int f0, int lane, TM (&v)[5]) {
  TM t[4];
  if (j < ny) {
    load_row<4>(g, j, f0, nx, t);
  } else {
#pragma unroll
    for (int k = 0; k < 4; ++k) t[k] = TM(0);
  }
#pragma unroll
  for (int k = 0; k < 4; ++k) v[k] = t[k];
  TM e = __shfl_down_sync(0xffffffffu, t[0], 1);
  if (lane == 31) e = (j < ny && f0 + 4 < nx) ? g.row(j)[f0 + 4] : TM(0);
  v[4] = e;
}

// C.b = P^T res (fine F), and the first sweep from zero: C.u = c C.b.  Two
// coarse columns a lane; coarse rows march upwards re-using the shared fine row.
template <class TM>
__device__ void mg_restrict(const Sched& s, const MgLevel<TM>& F, const TM* res, const MgLevel<TM>& C) {
  const Units un = make_units(C.nx, C.ny, 2, s.nw, 2);
  const Grid<const TM> gf{res, F.ld};
  const Grid<TM> gcb{C.b, C.ld}, gcu{C.u, C.ld};
  const TM c = (TM)kMgC;
  for (int u = s.w; u < un.nunits; u += s.nw) {
    int st, y0, y1;
    unit_bounds(un, u, C.ny, st, y0, y1);
    const int I0 = st * 64 + 2 * s.lane, f0 = 2 * I0;
    TM lo[5], mid[5], hi[5];
    mg_fine5(gf, F.nx, F.ny, 2 * y0, f0, s.lane, lo);
    for (int J = y0; J < y1; ++J) {
      mg_fine5(gf, F.nx, F.ny, 2 * J + 1, f0, s.lane, mid);
      mg_fine5(gf, F.nx, F.ny, 2 * J + 2, f0, s.lane, hi);
      TM bc[2], uc[2];
#pragma unroll
      for (int q = 0; q < 2; ++q) {  // coarse column I0 + q: fine columns f0 + 2q + {0, 1, 2}
        const int w = 2 * q, m = w + 1, e = w + 2;
        const TM s1 = ((mid[w] + mid[e]) + lo[m]) + hi[m];
        const TM s2 = ((lo[w] + lo[e]) + hi[w]) + hi[e];
        bc[q] = TM(0.25) * ((TM(4) * mid[m] + TM(2) * s1) + s2);
        uc[q] = c * bc[q];
      }
      store_row<2>(gcb, J, I0, C.nx, bc);
      store_row<2>(gcu, J, I0, C.nx, uc);
#pragma unroll
      for (int k = 0; k < 5; ++k) lo[k] = hi[k];
    }
  }
}

// Coarse values I0-1, I0, I0+1 of coarse row J for a lane whose fine columns
// are 2*I0 .. 2*I0+3 (I0 even): a 2-vector load, the first from the previous lane.
template <class TM>
__device__ __forceinline__ void mg_coarse3(const Grid<const TM>& g, int nx, int ny, int J, int I0, int lane,
                                           TM (&v)[3]) {
  TM t[2];
  if (J >= 0 && J < ny) {
    load_row<2>(g, J, I0, nx, t);
  } else {
    t[0] = TM(0);
    t[1] = TM(0);
  }
  TM w = __shfl_up_sync(0xffffffffu, t[1], 1);
  if (lane == 0) w = (J >= 0 && J < ny && I0 >= 1 && I0 - 1 < nx) ? g.row(J)[I0 - 1] : TM(0);
  v[0] = w;
  v[1] = t[0];
  v[2] = t[1];
}

// f += P e (coarse C, four fine columns a lane), rows marching upwards.
template <class TM>
__device__ void mg_prolong(const Sched& s, const MgLevel<TM>& F, TM* f, const MgLevel<TM>& C, const TM* e) {
  const Units un = make_units(F.nx, F.ny, 4, s.nw, 2);
  const Grid<const TM> gc{e, C.ld};
  const Grid<TM> gf{f, F.ld};
  for (int u = s.w; u < un.nunits; u += s.nw) {
    int st, y0, y1;
    unit_bounds(un, u, F.ny, st, y0, y1);
    const int f0 = st * 128 + 4 * s.lane, I0 = f0 / 2;
    // coarse rows J-1 (below) and J (at or above) of the current fine row
    int Jb = (y0 >> 1) - 1;
    TM cb[3], ca[3];
    mg_coarse3(gc, C.nx, C.ny, Jb, I0, s.lane, cb);
    mg_coarse3(gc, C.nx, C.ny, Jb + 1, I0, s.lane, ca);
    for (int j = y0; j < y1; ++j) {
      const int J = j >> 1;  // odd j: coarse row (j-1)/2 = J; even j: rows J-1 and J
      if (J - 1 != Jb) {
#pragma unroll
        for (int k = 0; k < 3; ++k) cb[k] = ca[k];
        Jb = J - 1;
        mg_coarse3(gc, C.nx, C.ny, J, I0, s.lane, ca);
      }
      TM v[4];
      if (j & 1) {  // odd fine row: coarse row J only
        v[0] = TM(0.5) * (ca[0] + ca[1]);
        v[1] = ca[1];
        v[2] = TM(0.5) * (ca[1] + ca[2]);
        v[3] = ca[2];
      } else {      // even fine row: coarse rows J-1 and J
        v[0] = TM(0.25) * ((cb[0] + cb[1]) + (ca[0] + ca[1]));
        v[1] = TM(0.5) * (cb[1] + ca[1]);
        v[2] = TM(0.25) * ((cb[1] + cb[2]) + (ca[1] + ca[2]));
        v[3] = TM(0.5) * (cb[2] + ca[2]);
      }
      TM cur[4];
      load_row<4>(Grid<const TM>{f, F.ld}, j, f0, F.nx, cur);
#pragma unroll
      for (int k = 0; k < 4; ++k) cur[k] += v[k];
      store_row<4>(gf, j, f0, F.nx, cur);
    }
  }
}

// Stencil operand row j of a V-cycle iterate, widened to binary64.
template <int V, class TM>
__device__ __forceinline__ void field_wide(const Grid<const TM>& g, int nx, int ny, int j, int x, int xs, int lane,
                                           FRow<V, double>& f) {
  if (j < 0 || j >= ny) {
    f.zero();
    return;
  }
  TM t[V];
  load_row<V>(g, j, x, nx, t);
#pragma unroll
  for (int k = 0; k < V; ++k) f.f[k] = mg_widen(t[k]);
  f.hl = (lane == 0 && xs >= 1 && xs - 1 < nx) ? mg_widen(g.row(j)[xs - 1]) : 0.0;
  f.hr = (lane == 31 && xs + 32 * V < nx) ? mg_widen(g.row(j)[xs + 32 * V]) : 0.0;
}

// Point-wise forms of the V-cycle's passes for the single-CTA levels: one
// thread a point, no warp-level march (at a few thousand points a pass the
// march's dependent row chain, not bandwidth, set the time).  Same operations
// in the same order as mg_stencil_pass, mg_restrict and mg_prolong.
template <class TM>
__device__ __forceinline__ TM tiny_at(const TM* g, int nx, int ny, int ld, int i, int j) {
  return (i < 0 || i >= nx || j < 0 || j >= ny) ? TM(0) : g[j * ld + i];
}

// f(i, j) at the thread's points of an nx x ny level: point p = j nx + i for
// p = threadIdx.x, + blockDim.x, ...; (i, j) advanced by the stride's row and
// column steps (two divisions a pass, none a point).
template <class F>
__device__ __forceinline__ void tiny_for(int nx, int ny, F&& f) {
  const int n = nx * ny;
  const int sj = (int)blockDim.x / nx, si = (int)blockDim.x - sj * nx;
  int j = (int)threadIdx.x / nx, i = (int)threadIdx.x - j * nx;
  for (int p = threadIdx.x; p < n; p += blockDim.x) {
    f(i, j);
    i += si;
    j += sj;
    if (i >= nx) {
      i -= nx;
      ++j;
    }
  }
}

template <class TM, bool JAC>
__device__ void tiny_stencil(const MgLevel<TM>& L, const TM* in, TM* out) {
  const TM c = (TM)kMgC;
  tiny_for(L.nx, L.ny, [&](int i, int j) {
    const TM C = in[j * L.ld + i];
    TM acc = TM(4) * C;
    acc -= tiny_at(in, L.nx, L.ny, L.ld, i - 1, j);
    acc -= tiny_at(in, L.nx, L.ny, L.ld, i + 1, j);
    acc -= tiny_at(in, L.nx, L.ny, L.ld, i, j - 1);
    acc -= tiny_at(in, L.nx, L.ny, L.ld, i, j + 1);
    const TM b = L.b[j * L.ld + i];
    out[j * L.ld + i] = JAC ? mg_fma(c, b - acc, C) : b - acc;
  });
}

// coarse C.b = P^T res, C.u = c C.b
template <class TM>
__device__ void tiny_restrict(const MgLevel<TM>& F, const TM* res, const MgLevel<TM>& C) {
  const TM c = (TM)kMgC;
  tiny_for(C.nx, C.ny, [&](int I, int J) {
    const int fi = 2 * I + 1, fj = 2 * J + 1;
    auto r = [&](int di, int dj) { return tiny_at(res, F.nx, F.ny, F.ld, fi + di, fj + dj); };
    const TM s1 = ((r(-1, 0) + r(1, 0)) + r(0, -1)) + r(0, 1);
    const TM s2 = ((r(-1, -1) + r(1, -1)) + r(-1, 1)) + r(1, 1);
    const TM bc = TM(0.25) * ((TM(4) * r(0, 0) + TM(2) * s1) + s2);
    C.b[J * C.ld + I] = bc;
    C.u[J * C.ld + I] = c * bc;
  });
}

// f += P e
template <class TM>
__device__ void tiny_prolong(const MgLevel<TM>& F, TM* f, const MgLevel<TM>& C, const TM* e) {
  tiny_for(F.nx, F.ny, [&](int i, int j) {
    auto ce = [&](int I, int J) { return tiny_at(e, C.nx, C.ny, C.ld, I, J); };
    TM v;
    if (j & 1) {
      const int J = j >> 1;
      v = (i & 1) ? ce(i >> 1, J) : TM(0.5) * (ce((i >> 1) - 1, J) + ce(i >> 1, J));
    } else {
      const int J = j >> 1;
      if (i & 1) {
        const int I = i >> 1;
        v = TM(0.5) * (ce(I, J - 1) + ce(I, J));
      } else {
        const int I = i >> 1;
        v = TM(0.25) * ((ce(I - 1, J - 1) + ce(I, J - 1)) + (ce(I - 1, J) + ce(I, J)));
      }
    }
    f[j * F.ld + i] += v;
  });
}

// The V-cycle from level `first` down to the coarsest and back with the
// point-wise passes, CTA barriers between them; returns the parity of the
// buffer that holds level `first`'s result (0: u, 1: v).
template <class TM>
__device__ int tiny_vcycle(const MgLevel<TM>* lv, int nlev, int first, int nu, int nu_c) {
  int cur[kMgMaxLevels] = {};  // 0: the level's iterate is in u, 1: in v
  auto it = [&](int l) -> TM* { return cur[l] ? lv[l].v : lv[l].u; };
  auto other = [&](int l) -> TM* { return cur[l] ? lv[l].u : lv[l].v; };
  auto jac = [&](int l) {
    tiny_stencil<TM, true>(lv[l], it(l), other(l));
    cur[l] ^= 1;
    __syncthreads();
  };
  cur[first] = 0;
  for (int l = first; l < nlev - 1; ++l) {
    for (int k = 1; k < nu; ++k) jac(l);
    tiny_stencil<TM, false>(lv[l], it(l), other(l));
    __syncthreads();
    tiny_restrict(lv[l], other(l), lv[l + 1]);
    __syncthreads();
    cur[l + 1] = 0;
  }
  for (int k = 1; k < nu_c; ++k) jac(nlev - 1);
  for (int l = nlev - 2; l >= first; --l) {
    tiny_prolong(lv[l], it(l), lv[l + 1], it(l + 1));
    __syncthreads();
    for (int k = 0; k < nu; ++k) jac(l);
  }
  return cur[first];
}

template <class TM>
struct Vcycle {
  int nlev, lsmall, nu, nu_c;  // as in PcgArgs
  const MgLevel<TM>* lv;       // the level descriptors, staged in shared memory
  GridTeam& tm;
  double* red;
  Sched grid, cta;
  Grid<const double> r;        // for the fused (r, z) of level 0's last sweep
  Acc64* dot;
  int cur[kMgMaxLevels];  // 0: the level's iterate is in u, 1: in v
  bool exec;              // this CTA runs the passes it meets (small levels: CTA 0 only)
  bool dot_done;          // (r, z) was accumulated (and the last barrier left to the caller)
  unsigned pc;            // pass counter: march direction

  __device__ TM* it(int l) const { return cur[l] ? lv[l].v : lv[l].u; }
  __device__ TM* other(int l) const { return cur[l] ? lv[l].u : lv[l].v; }
  __device__ bool small(int l) const { return l >= lsmall; }
  __device__ Sched sched(int l) {
    Sched s = small(l) ? cta : grid;
    s.rev = (pc++ & 1u) != 0u;
    return s;
  }
  // barrier after a pass at level l: grid-wide for big levels, CTA-wide for
  // small ones (which only CTA 0 runs)
  __device__ bool sync(int l) {
    if (small(l)) {
      __syncthreads();
      return true;
    }
    return tm.sync(red);
  }
  // a Jacobi sweep at level l; level 0's final sweep (last) accumulates
  // (r, z) and leaves its grid barrier to the caller's reduction
  __device__ bool jacobi(int l, bool last) {
    if (!exec) {
      cur[l] ^= 1;
      if (l == 0 && last && dot) dot_done = true;
      return true;
    }
    const Sched s = sched(l);
    Acc64 dummy;
    if (l == 0 && last && dot) {
      mg_stencil_pass<TM, true, true>(s, lv[l], it(l), other(l), r, *dot);
      dot_done = true;
      cur[l] ^= 1;
      if (small(l)) __syncthreads();
      return true;
    }
    mg_stencil_pass<TM, true, false>(s, lv[l], it(l), other(l), r, dummy);
    cur[l] ^= 1;
    return sync(l);
  }
  // sweeps 2..n of damped Jacobi (the first sweep, u = c b, came with b)
  __device__ bool sweeps(int l, int n, bool final_level0) {
    for (int k = 1; k < n; ++k)
      if (!jacobi(l, final_level0 && k == n - 1)) return false;
    return true;
  }
  __device__ bool down(int l) {  // pre-smoothing, residual, restriction into l+1
    if (!sweeps(l, nu, false)) return false;
    if (exec) {
      Acc64 dummy;
      mg_stencil_pass<TM, false, false>(sched(l), lv[l], it(l), other(l), r, dummy);
      if (!sync(l)) return false;
      mg_restrict(sched(l), lv[l], other(l), lv[l + 1]);
      if (!sync(l)) return false;
    }
    cur[l + 1] = 0;
    return true;
  }
  __device__ bool up(int l) {  // prolongation from l+1, then nu post-smoothing sweeps
    if (exec) {
      mg_prolong(sched(l), lv[l], it(l), lv[l + 1], it(l + 1));
      if (!sync(l)) return false;
    }
    for (int k = 0; k < nu; ++k)
      if (!jacobi(l, l == 0 && k == nu - 1)) return false;
    return true;
  }
  // One V-cycle; level 0's b and u = c b are in place.  Returns false when
  // the solve must stop (abort or barrier timeout).
  // start0: the buffer (0: u, 1: v) that holds level 0's first sweep.
  __device__ bool run(int start0 = 0) {
    const int L = nlev;
    cur[0] = start0;
    dot_done = false;
    const int big_end = min(lsmall, L - 1);  // levels [0, big_end) restrict grid-wide
    exec = true;
    for (int l = 0; l < big_end; ++l)
      if (!down(l)) return false;
    if (lsmall >= L) {  // the coarsest level is big
      if (!sweeps(L - 1, nu_c, L == 1)) return false;
    } else {
      // CTA 0 alone runs the levels [big_end, L) with the point-wise passes
      // (the warp march's dependent row chain, not bandwidth, sets the time at
      // these sizes); every CTA knows where level big_end's result ends
      if (blockIdx.x == 0) (void)tiny_vcycle<TM>(lv, L, big_end, nu, nu_c);
      cur[big_end] = (big_end < L - 1 ? 2 * nu - 1 : nu_c - 1) & 1;
      if (!tm.sync(red)) return false;  // publishes CTA 0's levels
    }
    for (int l = big_end - 1; l >= 0; --l)
      if (!up(l)) return false;
    return true;
  }
};

}  // namespace lap5
