// common.cuh -- device building blocks shared by the lap5cg kernels:
// element storage (binary64 / binary32 / bf16), lane-vector loads and stores,
// the 5-point stencil on a warp strip, Dot2 accumulation, and the persistent
// kernel's grid barrier and deterministic grid reduction.
//
// Target: sm_103a (GB300).  No tensor cores: the 5-point stencil is not a
// dense contraction.
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <cooperative_groups.h>
#include <stdint.h>
#include <type_traits>

#include "../../include/lap5cg.h"

namespace lap5 {

// ---------------------------------------------------------------------------
// Storage types.  bf16 is kept as raw 16-bit words; widening to binary32 is a
// shift, narrowing uses the hardware round-to-nearest-even conversion.
// ---------------------------------------------------------------------------
struct bf16s { uint16_t bits; };

template <class T> struct Math;                       // arithmetic type per storage type
template <> struct Math<double> { using type = double; };
template <> struct Math<float> { using type = float; };
template <> struct Math<bf16s> { using type = float; };

__device__ __forceinline__ float bf_widen(uint16_t h) { return __uint_as_float(((uint32_t)h) << 16); }
__device__ __forceinline__ uint16_t bf_narrow(float f) {
  __nv_bfloat16 h = __float2bfloat16_rn(f);
  return *reinterpret_cast<uint16_t*>(&h);
}

template <class M, class T> __device__ __forceinline__ M to_math(T v);
template <> __device__ __forceinline__ double to_math<double, double>(double v) { return v; }
template <> __device__ __forceinline__ float to_math<float, float>(float v) { return v; }
template <> __device__ __forceinline__ float to_math<float, bf16s>(bf16s v) { return bf_widen(v.bits); }

template <class T, class M> __device__ __forceinline__ T from_math(M v);
template <> __device__ __forceinline__ double from_math<double, double>(double v) { return v; }
template <> __device__ __forceinline__ float from_math<float, float>(float v) { return v; }
template <> __device__ __forceinline__ bf16s from_math<bf16s, float>(float v) { return bf16s{bf_narrow(v)}; }

// Fused multiply-add in the arithmetic type (never promotes binary32 to binary64).
__device__ __forceinline__ double fmx(double a, double b, double c) { return __fma_rn(a, b, c); }
__device__ __forceinline__ float fmx(float a, float b, float c) { return __fmaf_rn(a, b, c); }

// Round a value of the arithmetic type to the storage type and back (identity
// unless the storage is narrower, e.g. bf16).
template <class T> __device__ __forceinline__ float quantize(float v) { return v; }
template <> __device__ __forceinline__ float quantize<bf16s>(float v) { return bf_widen(bf_narrow(v)); }

// A strided grid view: element (i, j) at ptr[j*ld + i].
template <class T> struct Grid {
  T* ptr;
  int ld;
  __device__ __forceinline__ T* row(int j) const { return ptr + (size_t)j * (size_t)ld; }
};

// ---------------------------------------------------------------------------
// Lane layout of a warp strip of 32*V columns starting at xs.  A lane owns V
// columns in G = V / W groups of W = min(V, 4) consecutive columns; group g of
// lane l starts at column xs + 32*W*g + W*l.  With V <= 4 this is one group of
// V consecutive columns; with V = 8 (binary32) a lane holds two 16-byte
// vectors 128 columns apart, so every lane-vector access of the warp covers
// 512 contiguous bytes (conflict-free in shared memory, full sectors in HBM).
// ---------------------------------------------------------------------------
template <int V> struct Lanes {
  static constexpr int W = V > 4 ? 4 : V;
  static constexpr int G = V / W;
  static constexpr int GS = 32 * W;  // column distance between a lane's groups
  // column of the lane's element k relative to its first column
  __host__ __device__ static constexpr int col(int k) { return (k / W) * GS + (k % W); }
  // one past the lane's last column relative to its first column
  static constexpr int span = (G - 1) * GS + W;
  __host__ __device__ static constexpr int first(int xs, int lane) { return xs + lane * W; }
};

// ---------------------------------------------------------------------------
// Lane-vector IO: VecIO<W> moves W consecutive columns x .. x+W-1 of a row.
// The vector path needs the row start 16-byte aligned for binary64 / binary32
// (8-byte for bf16 with V = 4) and ld a multiple of V: then a vector that
// straddles nx stays inside the row's ld elements and is masked after the load.
// ---------------------------------------------------------------------------
template <int V, class T> struct VecIO;

template <> struct VecIO<2, double> {
  __device__ __forceinline__ static void load(const double* p, double (&v)[2]) {
    double2 t = *reinterpret_cast<const double2*>(p);
    v[0] = t.x; v[1] = t.y;
  }
  __device__ __forceinline__ static void store(double* p, const double (&v)[2]) {
    *reinterpret_cast<double2*>(p) = make_double2(v[0], v[1]);
  }
};
template <> struct VecIO<2, float> {
  __device__ __forceinline__ static void load(const float* p, float (&v)[2]) {
    float2 t = *reinterpret_cast<const float2*>(p);
    v[0] = t.x; v[1] = t.y;
  }
  __device__ __forceinline__ static void store(float* p, const float (&v)[2]) {
    *reinterpret_cast<float2*>(p) = make_float2(v[0], v[1]);
  }
};
template <> struct VecIO<2, bf16s> {
  __device__ __forceinline__ static void load(const bf16s* p, float (&v)[2]) {
    const uint32_t t = *reinterpret_cast<const uint32_t*>(p);
    v[0] = __uint_as_float(t << 16); v[1] = __uint_as_float(t & 0xffff0000u);
  }
  __device__ __forceinline__ static void store(bf16s* p, const float (&v)[2]) {
    *reinterpret_cast<uint32_t*>(p) = (uint32_t)bf_narrow(v[0]) | ((uint32_t)bf_narrow(v[1]) << 16);
  }
};
template <> struct VecIO<4, float> {
  __device__ __forceinline__ static void load(const float* p, float (&v)[4]) {
    float4 t = *reinterpret_cast<const float4*>(p);
    v[0] = t.x; v[1] = t.y; v[2] = t.z; v[3] = t.w;
  }
  __device__ __forceinline__ static void store(float* p, const float (&v)[4]) {
    *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], v[3]);
  }
};
template <> struct VecIO<4, bf16s> {
  __device__ __forceinline__ static void load(const bf16s* p, float (&v)[4]) {
    uint2 t = *reinterpret_cast<const uint2*>(p);
    v[0] = __uint_as_float(t.x << 16); v[1] = __uint_as_float(t.x & 0xffff0000u);
    v[2] = __uint_as_float(t.y << 16); v[3] = __uint_as_float(t.y & 0xffff0000u);
  }
  __device__ __forceinline__ static void store(bf16s* p, const float (&v)[4]) {
    uint2 t;
    t.x = (uint32_t)bf_narrow(v[0]) | ((uint32_t)bf_narrow(v[1]) << 16);
    t.y = (uint32_t)bf_narrow(v[2]) | ((uint32_t)bf_narrow(v[3]) << 16);
    *reinterpret_cast<uint2*>(p) = t;
  }
};
template <> struct VecIO<4, double> {
  __device__ __forceinline__ static void load(const double* p, double (&v)[4]) {
    const double2 a = reinterpret_cast<const double2*>(p)[0];
    const double2 b = reinterpret_cast<const double2*>(p)[1];
    v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y;
  }
  __device__ __forceinline__ static void store(double* p, const double (&v)[4]) {
    reinterpret_cast<double2*>(p)[0] = make_double2(v[0], v[1]);
    reinterpret_cast<double2*>(p)[1] = make_double2(v[2], v[3]);
  }
};

// V = 1: plain scalar accesses (rows without 16-byte alignment).
template <class T> struct VecIO<1, T> {
  template <class M>
  __device__ __forceinline__ static void load(const T* p, M (&v)[1]) { v[0] = to_math<M, T>(p[0]); }
  template <class M>
  __device__ __forceinline__ static void store(T* p, const M (&v)[1]) { p[0] = from_math<T, M>(v[0]); }
};

// Load the lane's V values of row j; columns >= nx read as 0.  x < ld is
// guaranteed by the caller (x is a lane column inside an ld-aligned row).
// Load W consecutive values at p (column x); columns >= nx read as 0.
template <int W, class U, class M>
__device__ __forceinline__ void load_group(const U* p, int x, int nx, M (&v)[W]) {
  if (x < nx) {
    VecIO<W, U>::load(p, v);
    if (x + W > nx) {
#pragma unroll
      for (int k = 0; k < W; ++k)
        if (x + k >= nx) v[k] = M(0);
    }
  } else {
#pragma unroll
    for (int k = 0; k < W; ++k) v[k] = M(0);
  }
}

// Load the lane's V values of row j (lane layout above; x = the lane's first
// column); columns >= nx read as 0.
template <int V, class T, class M>
__device__ __forceinline__ void load_row(const Grid<T>& g, int j, int x, int nx, M (&v)[V]) {
  using U = typename std::remove_const<T>::type;
  using L = Lanes<V>;
  if constexpr (L::G == 1) {
    load_group<V, U, M>(g.row(j) + x, x, nx, v);
  } else {
#pragma unroll
    for (int gi = 0; gi < L::G; ++gi) {
      M t[L::W];
      const int xg = x + gi * L::GS;
      load_group<L::W, U, M>(g.row(j) + xg, xg, nx, t);
#pragma unroll
      for (int k = 0; k < L::W; ++k) v[gi * L::W + k] = t[k];
    }
  }
}

// Store the lane's V values of row j; columns >= nx are not written.
template <int W, class T, class M>
__device__ __forceinline__ void store_group(T* p, int x, int nx, const M (&v)[W]) {
  if (x + W <= nx) {
    VecIO<W, T>::store(p, v);
  } else if (x < nx) {
#pragma unroll
    for (int k = 0; k < W; ++k)
      if (x + k < nx) p[k] = from_math<T, M>(v[k]);
  }
}

template <int V, class T, class M>
__device__ __forceinline__ void store_row(const Grid<T>& g, int j, int x, int nx, const M (&v)[V]) {
  using L = Lanes<V>;
  if constexpr (L::G == 1) {
    store_group<V, T, M>(g.row(j) + x, x, nx, v);
  } else {
#pragma unroll
    for (int gi = 0; gi < L::G; ++gi) {
      M t[L::W];
#pragma unroll
      for (int k = 0; k < L::W; ++k) t[k] = v[gi * L::W + k];
      const int xg = x + gi * L::GS;
      store_group<L::W, T, M>(g.row(j) + xg, xg, nx, t);
    }
  }
}

// Scalar load for a halo column; 0 outside [0, nx).
template <class T, class M>
__device__ __forceinline__ M load_one(const Grid<T>& g, int j, int x, int nx) {
  using U = typename std::remove_const<T>::type;
  if (x < 0 || x >= nx) return M(0);
  return to_math<M, U>(g.row(j)[x]);
}

// ---------------------------------------------------------------------------
// Field rows.  A "field" is the vector the stencil is applied to; a warp keeps
// three consecutive field rows (S, C, N) in registers.  hl / hr are the field
// values at the strip's left / right halo columns (meaningful on lane 0 / 31).
// ---------------------------------------------------------------------------
template <int V, class M> struct FRow {
  M f[V];
  M hl, hr;
  __device__ __forceinline__ void zero() {
#pragma unroll
    for (int k = 0; k < V; ++k) f[k] = M(0);
    hl = M(0); hr = M(0);
  }
};

__device__ __forceinline__ double shfl_up1(double v) { return __shfl_up_sync(0xffffffffu, v, 1); }
__device__ __forceinline__ float shfl_up1(float v) { return __shfl_up_sync(0xffffffffu, v, 1); }
__device__ __forceinline__ double shfl_dn1(double v) { return __shfl_down_sync(0xffffffffu, v, 1); }
__device__ __forceinline__ float shfl_dn1(float v) { return __shfl_down_sync(0xffffffffu, v, 1); }

// y = A f on the centre row: the Sec. II-B mask in the fixed add order
// 4*C - W - E - S - N.  4*C is exact, so contracting the first subtraction
// into a fused multiply-add does not change the result.  Whole-warp call.
template <int V, class M>
__device__ __forceinline__ void stencil_row(const FRow<V, M>& S, const FRow<V, M>& C, const FRow<V, M>& N,
                                            int lane, M (&y)[V]) {
  using L = Lanes<V>;
  constexpr int W = L::W;
#pragma unroll
  for (int gi = 0; gi < L::G; ++gi) {
    M left, right;
    if constexpr (L::G == 1) {
      left = shfl_up1(C.f[V - 1]);
      right = shfl_dn1(C.f[0]);
    } else {
      // west of lane 0's group gi is lane 31's group gi-1; east of lane 31's
      // group gi is lane 0's group gi+1 (rotating shuffles)
      const M wv = (lane == 31 && gi > 0) ? C.f[gi * W - 1] : C.f[gi * W + W - 1];
      const M ev = (lane == 0 && gi < L::G - 1) ? C.f[(gi + 1) * W] : C.f[gi * W];
      left = __shfl_sync(0xffffffffu, wv, (lane + 31) & 31);
      right = __shfl_sync(0xffffffffu, ev, (lane + 1) & 31);
    }
    if (gi == 0 && lane == 0) left = C.hl;
    if (gi == L::G - 1 && lane == 31) right = C.hr;
#pragma unroll
    for (int q = 0; q < W; ++q) {
      const int k = gi * W + q;
      const M w = (q == 0) ? left : C.f[k - 1];
      const M e = (q == W - 1) ? right : C.f[k + 1];
      M acc = M(4) * C.f[k];
      acc -= w;
      acc -= e;
      acc -= S.f[k];
      acc -= N.f[k];
      y[k] = acc;
    }
  }
}

// Accumulate (a, b) over the lane's valid elements: element k is valid when
// its column offset Lanes<V>::col(k) < ncols (ncols = nx - the lane's first
// column).  A single uniform branch for lanes whose columns are all inside.
template <int V, class Acc, class M>
__device__ __forceinline__ void acc_dot(Acc& acc, int j, const M (&a)[V], const M (&b)[V], int ncols) {
  (void)j;  // the row index matters to the exact accumulator only
  if (ncols >= Lanes<V>::span) {
    acc.add_block(a, b);
  } else if (ncols > 0) {
    M am[V];
#pragma unroll
    for (int k = 0; k < V; ++k) am[k] = Lanes<V>::col(k) < ncols ? a[k] : M(0);
    acc.add_block(am, b);
  }
}

// ---------------------------------------------------------------------------
// Dot-product accumulators.  binary64: plain fused multiply-add.  binary32:
// Dot2 of Ogita, Rump & Oishi (SIAM J. Sci. Comput. 2005) -- TwoProduct by
// fmaf, TwoSum by Knuth -- carried per thread as (s, c); the cross-thread
// reduction then runs in binary64 on s + c.
// ---------------------------------------------------------------------------
struct Acc64 {
  double s = 0.0;
  __device__ __forceinline__ void add(double a, double b) { s = __fma_rn(a, b, s); }
  template <int V>
  __device__ __forceinline__ void add_block(const double (&a)[V], const double (&b)[V]) {
#pragma unroll
    for (int k = 0; k < V; ++k) s = __fma_rn(a[k], b[k], s);
  }
  __device__ __forceinline__ double value() const { return s; }
};
struct Acc32 {
  float s = 0.f, c = 0.f;
  // The _rn intrinsics are never contracted into fused multiply-adds, which
  // the error-free transformations rely on.
  __device__ __forceinline__ void add(float a, float b) {
    const float h = __fmul_rn(a, b);
    const float l = __fmaf_rn(a, b, -h);
    const float x = __fadd_rn(s, h);
    const float zz = __fsub_rn(x, s);
    const float e = __fadd_rn(__fsub_rn(s, __fsub_rn(x, zz)), __fsub_rn(h, zz));
    s = x;
    c = __fadd_rn(c, __fadd_rn(e, l));
  }
  // A lane's V products of one row: summed with fused multiply-adds, and the
  // partial added to (s, c) with TwoSum.  The compensation then acts between
  // row blocks; within a block the error is at most (V-1) roundings of the
  // block's partial sums.  About a quarter of Dot2's instructions per element.
  template <int V>
  __device__ __forceinline__ void add_block(const float (&a)[V], const float (&b)[V]) {
    float p = __fmul_rn(a[0], b[0]);
#pragma unroll
    for (int k = 1; k < V; ++k) p = __fmaf_rn(a[k], b[k], p);
    const float x = __fadd_rn(s, p);
    const float zz = __fsub_rn(x, s);
    const float e = __fadd_rn(__fsub_rn(s, __fsub_rn(x, zz)), __fsub_rn(p, zz));
    s = x;
    c = __fadd_rn(c, e);
  }
  __device__ __forceinline__ double value() const { return (double)s + (double)c; }
};
template <class M> struct AccOf;
template <> struct AccOf<double> { using type = Acc64; };
template <> struct AccOf<float> { using type = Acc32; };

// ---------------------------------------------------------------------------
// Control block in the workspace (zeroed by the host before each launch).
// ---------------------------------------------------------------------------
constexpr int kMaxCtas = 2048;     // partial-sum slots per parity
constexpr int kMaxVals = 4;        // reduced values per barrier

constexpr int kExactLimbs = 67;  // exact accumulator: 32-bit digits over 2^-1074 .. 2^1024, plus carry room
constexpr int kExactSlots = 2;   // exact dot products per reduction

struct Ctl {
  unsigned long long bar;          // monotonic arrival counter
  int abort;                       // nonzero: every CTA leaves at its next check
  int status;                      // first error recorded (0 = none)
  int pad[12];
  // exact (reproducible) dot products: the solve's accumulators, three
  // buffers used in turn by successive exact reductions
  unsigned long long xacc[3][kExactSlots][kExactLimbs];
  unsigned xbad[3][kExactSlots];
  unsigned xpad[2];
  double part[2][kMaxCtas][kMaxVals];  // per-CTA partials, double-buffered by barrier parity
};

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ unsigned long long ld_acquire_u64(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ int ld_relaxed_i32(const int* p) {
  int v;
  asm volatile("ld.relaxed.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ void record_error(Ctl* ctl, int code) {
  atomicCAS(&ctl->status, 0, code);
  __threadfence();
  atomicExch(&ctl->abort, 1);
}

// Grid-wide reduction of NV values with a barrier.  Every thread passes its
// per-thread contributions in v[]; on return every thread of every CTA holds
// the same totals in out[] (fixed summation order: lanes, warps, then CTA
// slots 0..G-1), or the function returns false when the solve must stop
// (abort flag or barrier timeout).  Needs blockDim.x / 32 <= 32 and
// kMaxVals * 32 doubles of shared scratch (red).
template <int NV>
__device__ __forceinline__ bool grid_reduce(Ctl* ctl, unsigned long long& epoch, const double (&v)[NV],
                                            double (&out)[NV], double* red, long long timeout_ns) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  double t[NV];
#pragma unroll
  for (int k = 0; k < NV; ++k) {
    double s = v[k];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    t[k] = s;
  }
  __shared__ int s_go;
  if (lane == 0) {
#pragma unroll
    for (int k = 0; k < NV; ++k) red[warp * kMaxVals + k] = t[k];
  }
  __syncthreads();
  const int par = (int)(epoch & 1ull);
  if (warp == 0) {
#pragma unroll
    for (int k = 0; k < NV; ++k) {
      double s = lane < nwarps ? red[lane * kMaxVals + k] : 0.0;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
      if (lane == 0) ctl->part[par][blockIdx.x][k] = s;
    }
    if (lane == 0) {
      int go = 1;
      __threadfence();
      atomicAdd(&ctl->bar, 1ull);
      const unsigned long long target = (epoch + 1ull) * (unsigned long long)gridDim.x;
      const unsigned long long t0 = global_ns();
      unsigned spins = 0;
      while (ld_acquire_u64(&ctl->bar) < target) {
        if ((++spins & 7u) == 0u) {  // each poll is an L2 round trip: check the clock often
          if (ld_relaxed_i32(&ctl->abort)) { go = 0; break; }
          if ((long long)(global_ns() - t0) > timeout_ns) {
            record_error(ctl, LAP5CG_ERR_SYNC_TIMEOUT);
            go = 0;
            break;
          }
        }
      }
      if (go && ld_relaxed_i32(&ctl->abort)) go = 0;
      __threadfence();
      s_go = go;
    }
    __syncwarp();
    // sum the CTA slots in a fixed order (identical in every CTA)
#pragma unroll
    for (int k = 0; k < NV; ++k) {
      double s = 0.0;
      for (int c = lane; c < (int)gridDim.x; c += 32) s += *((volatile double*)&ctl->part[par][c][k]);
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
      if (lane == 0) red[32 * kMaxVals + k] = s;
    }
  }
  __syncthreads();
  ++epoch;
  const bool go = s_go != 0;
#pragma unroll
  for (int k = 0; k < NV; ++k) out[k] = red[32 * kMaxVals + k];
  __syncthreads();  // red is reused by the next call
  return go;
}

// Plain grid barrier (no values), same protocol as grid_reduce.
__device__ __forceinline__ bool grid_sync(Ctl* ctl, unsigned long long& epoch, double* red, long long timeout_ns) {
  double v[1] = {0.0}, o[1];
  return grid_reduce<1>(ctl, epoch, v, o, red, timeout_ns);
}

// Row march over one warp unit [y0, y1) of a strip, in either direction.
// field(j, FRow&) fills the stencil operand of row j (zeros outside [0, ny));
// load(j, D&) loads the row's other operands; finish(j, d, S, C, N) consumes
// row j with its south (j-1), centre and north (j+1) field rows.  One row of
// look-ahead: the loads of the next row are issued before the current row is
// finished.  Whole-warp call.
template <int V, class M, class D, class FieldF, class LoadF, class FinishF>
__device__ __forceinline__ void march(int y0, int y1, bool rev, FieldF& field, LoadF& load, FinishF& finish) {
  if (y0 >= y1) return;
  const int step = rev ? -1 : 1;
  int j = rev ? y1 - 1 : y0;
  const int jend = rev ? y0 - 1 : y1;
  FRow<V, M> fB, fC;
  D dC;
  field(j - step, fB);
  field(j, fC);
  load(j, dC);
  for (; j != jend; j += step) {
    FRow<V, M> fA;
    D dA;
    field(j + step, fA);
    if (j + step != jend) load(j + step, dA);
    if (!rev) finish(j, dC, fB, fC, fA);
    else finish(j, dC, fA, fC, fB);
    fB = fC;
    fC = fA;
    dC = dA;
  }
}

// Same traversal without a stencil operand (element-wise passes).
template <class D, class LoadF, class FinishF>
__device__ __forceinline__ void stream_rows(int y0, int y1, bool rev, LoadF& load, FinishF& finish) {
  if (y0 >= y1) return;
  const int step = rev ? -1 : 1;
  int j = rev ? y1 - 1 : y0;
  const int jend = rev ? y0 - 1 : y1;
  D dC;
  load(j, dC);
  for (; j != jend; j += step) {
    D dA;
    if (j + step != jend) load(j + step, dA);
    finish(j, dC);
    dC = dA;
  }
}

// Geometry of the warp-unit decomposition of an nx-by-ny grid.
struct Units {
  int ns;        // strips of 32*V columns
  int nseg;      // row segments per strip
  int seg_rows;  // rows per segment (the last one may be shorter)
  int nunits;    // ns * nseg
};

// Units for W warps: as many row segments per strip as there are warps per
// strip, but no segment shorter than min_rows (halo rows cost two extra row
// loads per segment); segments rebalanced to equal height.
// row_align > 1: segment heights are multiples of row_align (segments start at
// multiples of it).
__host__ __device__ inline Units make_units(int nx, int ny, int V, long long W, int min_rows, int row_align = 1) {
  Units u;
  u.ns = (nx + 32 * V - 1) / (32 * V);
  long long nseg = W / u.ns;
  if (nseg < 1) nseg = 1;
  if (nseg > ny) nseg = ny;
  int L = (int)((ny + nseg - 1) / nseg);
  if (L < min_rows) L = min_rows < ny ? min_rows : ny;
  nseg = (ny + L - 1) / L;
  L = (int)((ny + nseg - 1) / nseg);
  if (row_align > 1) {
    L = (L + row_align - 1) / row_align * row_align;
    nseg = (ny + L - 1) / L;
  }
  u.nseg = (int)nseg;
  u.seg_rows = L;
  u.nunits = (int)((long long)u.ns * nseg);
  return u;
}

// Shared scratch every solve body needs: per-warp partials (32 x kMaxVals),
// totals (kMaxVals) and, for cluster teams, the CTA partial by parity
// (2 x kMaxVals).
constexpr int kRedDoubles = 35 * kMaxVals;

// A team is the set of CTAs that solve one system together.
//  GridTeam: every CTA of a cooperative launch; the barrier is the bounded
//  spin in grid_reduce.
struct GridTeam {
  Ctl* ctl;
  long long timeout_ns;
  unsigned long long epoch;
  unsigned long long* xs = nullptr;  // CTA exact accumulators [kExactSlots][kExactLimbs] (shared memory)
  unsigned* xsb = nullptr;           // their non-finite flags
  unsigned xepoch = 0;               // exact reductions so far
  __device__ __forceinline__ int rank() const { return (int)blockIdx.x; }
  __device__ __forceinline__ int size() const { return (int)gridDim.x; }
  template <int NV>
  __device__ __forceinline__ bool reduce(const double (&v)[NV], double (&o)[NV], double* red) {
    return grid_reduce<NV>(ctl, epoch, v, o, red, timeout_ns);
  }
  __device__ __forceinline__ bool sync(double* red) { return grid_sync(ctl, epoch, red, timeout_ns); }
};

//  ClusterTeam: the CTAs of one thread-block cluster.  The barrier is the
//  hardware cluster barrier, whose arrive has release and whose wait has
//  acquire semantics at cluster scope: global-memory halo values written by one
//  CTA before the barrier are visible to the cluster's other CTAs after it.
//  Partial sums move through distributed shared memory.  No spin-wait, so
//  nothing to time out.
struct ClusterTeam {
  unsigned long long epoch;
  __device__ __forceinline__ int rank() const { return (int)cooperative_groups::this_cluster().block_rank(); }
  __device__ __forceinline__ int size() const { return (int)cooperative_groups::this_cluster().num_blocks(); }
  __device__ __forceinline__ void barrier() { cooperative_groups::this_cluster().sync(); }
  template <int NV>
  __device__ __forceinline__ bool reduce(const double (&v)[NV], double (&out)[NV], double* red) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    const int par = (int)(epoch & 1ull);
    double* slot = red + 33 * kMaxVals + par * kMaxVals;
#pragma unroll
    for (int k = 0; k < NV; ++k) {
      double s = v[k];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
      if (lane == 0) red[warp * kMaxVals + k] = s;
    }
    __syncthreads();
    if (warp == 0) {
#pragma unroll
      for (int k = 0; k < NV; ++k) {
        double s = lane < nwarps ? red[lane * kMaxVals + k] : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (lane == 0) slot[k] = s;
      }
    }
    barrier();
    if (warp == 0) {
      auto cl = cooperative_groups::this_cluster();
      const int n = (int)cl.num_blocks();
#pragma unroll
      for (int k = 0; k < NV; ++k) {
        double s = 0.0;
        if (lane < n) s = *cl.map_shared_rank(slot + k, (unsigned)lane);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (lane == 0) red[32 * kMaxVals + k] = s;
      }
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < NV; ++k) out[k] = red[32 * kMaxVals + k];
    __syncthreads();
    ++epoch;
    return true;
  }
  __device__ __forceinline__ bool sync(double*) {
    barrier();
    ++epoch;
    return true;
  }
};

__device__ __forceinline__ void unit_bounds(const Units& u, int unit, int ny, int& strip, int& y0, int& y1) {
  strip = unit % u.ns;
  const int seg = unit / u.ns;
  y0 = seg * u.seg_rows;
  y1 = min(ny, y0 + u.seg_rows);
}

}  // namespace lap5
