// stencil.cu -- lap5_apply: y = A x for the 5-point Dirichlet Laplacian
// (arxiv 1803.03797, Sec. II-B mask), binary64 / binary32 / bf16 storage.
//
// One warp computes R consecutive rows of one strip of 32 V columns (the lane
// layout of the solver passes).  It issues the loads of all R + 2 operand rows
// before finishing the first output row, so no load waits on another; the
// rows shared with the warps above and below come from L1/L2, and x is read
// from HBM about once.  Not persistent, no grid barrier: enough independent
// warps keep the loads in flight.  (Measured at 8192^2 binary32: 5.6 TB/s,
// against 4.2 TB/s for a row march with one row of look-ahead.)
#include "common.cuh"
#include "launch.h"

namespace lap5 {

constexpr int kApplyRows = 2;  // output rows a warp
constexpr int kApplyWarps = 8;

template <class T, int V, int R>
__global__ void __launch_bounds__(32 * kApplyWarps) k_lap5_apply(int nx, int ny, Grid<const T> x, Grid<T> y, int ns) {
  using M = typename Math<T>::type;
  const int lane = threadIdx.x & 31;
  const int s = blockIdx.x % ns;
  const int jb = (blockIdx.x / ns) * (kApplyWarps * R) + (int)(threadIdx.x >> 5) * R;
  if (jb >= ny) return;
  const int xs = s * 32 * V, xl = Lanes<V>::first(xs, lane);
  FRow<V, M> f[R + 2];  // operand rows jb - 1 .. jb + R
#pragma unroll
  for (int k = 0; k < R + 2; ++k) {
    const int j = jb - 1 + k;
    if (j < 0 || j >= ny) {
      f[k].zero();
      continue;
    }
    load_row<V>(x, j, xl, nx, f[k].f);
    f[k].hl = (lane == 0) ? load_one<const T, M>(x, j, xs - 1, nx) : M(0);
    f[k].hr = (lane == 31) ? load_one<const T, M>(x, j, xs + 32 * V, nx) : M(0);
  }
#pragma unroll
  for (int k = 0; k < R; ++k) {
    if (jb + k < ny) {
      M yv[V];
      stencil_row<V>(f[k], f[k + 1], f[k + 2], lane, yv);
      store_row<V>(y, jb + k, xl, nx, yv);
    }
  }
}

// bf16 storage: sixteen columns a lane in two 16-byte vectors 256 columns
// apart (a warp strip is 512 columns; every warp access covers 512 contiguous
// bytes), processed one vector at a time so that at most 85 registers are
// live (three CTAs an SM); binary32 arithmetic in the fixed add order, result
// rounded to nearest even two columns a conversion.  Needs ld a multiple of 8
// and 16-byte aligned rows; a vector that straddles nx stays inside the row's
// ld elements and is masked.  Kept apart from the generic lane layout:
// measured at 8192^2 it moves 4.8 TB/s, where one vector a lane reaches 4.5,
// two vectors processed together 4.3 (more registers live), four columns a
// lane (8-byte accesses) 3.0, and packed f32x2 arithmetic does not help (the
// arithmetic is not the limit).
constexpr int kBfRows = 2;    // output rows a warp
constexpr int kBfGroups = 2;  // 16-byte vectors a lane

__device__ __forceinline__ uint32_t bf_pack2(float lo, float hi) {
  const __nv_bfloat162 h = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<const uint32_t*>(&h);
}
__device__ __forceinline__ float bf_lo(uint32_t w) { return __uint_as_float(w << 16); }
__device__ __forceinline__ float bf_hi(uint32_t w) { return __uint_as_float(w & 0xffff0000u); }

__global__ void __launch_bounds__(32 * kApplyWarps, 3) k_lap5_apply_bf16x16(int nx, int ny, int ld,
                                                                            const uint16_t* __restrict__ x,
                                                                            uint16_t* __restrict__ y, int ns) {
  constexpr int R = kBfRows, G = kBfGroups;
  const int lane = threadIdx.x & 31;
  const int s = blockIdx.x % ns;
  const int jb = (blockIdx.x / ns) * (kApplyWarps * R) + (int)(threadIdx.x >> 5) * R;
  if (jb >= ny) return;
  const int xs = s * 256 * G;
  uint4 raw[R + 2][G];  // operand rows jb - 1 .. jb + R, packed
#pragma unroll
  for (int k = 0; k < R + 2; ++k) {
    const int j = jb - 1 + k;
#pragma unroll
    for (int g = 0; g < G; ++g) {
      const int xc = xs + 256 * g + 8 * lane;
      raw[k][g] = (j >= 0 && j < ny && xc < nx) ? *reinterpret_cast<const uint4*>(x + (size_t)j * ld + xc)
                                                : make_uint4(0u, 0u, 0u, 0u);
    }
  }
#pragma unroll
  for (int k = 0; k < R; ++k) {
    const int j = jb + k;
    if (j >= ny) break;
    // the strip's halo columns (lanes 0 and 31)
    const float hl = (lane == 0 && xs >= 1) ? bf_widen(x[(size_t)j * ld + xs - 1]) : 0.f;
    const float hr = (lane == 31 && xs + 256 * G < nx) ? bf_widen(x[(size_t)j * ld + xs + 256 * G]) : 0.f;
#pragma unroll
    for (int g = 0; g < G; ++g) {
      const int xc = xs + 256 * g + 8 * lane;
      float S[8], C[8], N[8], Y[8];
      const uint4 rs = raw[k][g], rc = raw[k + 1][g], rn = raw[k + 2][g];
      const uint32_t ws[4] = {rs.x, rs.y, rs.z, rs.w}, wc[4] = {rc.x, rc.y, rc.z, rc.w},
                     wn[4] = {rn.x, rn.y, rn.z, rn.w};
#pragma unroll
      for (int m = 0; m < 4; ++m) {
        S[2 * m] = bf_lo(ws[m]);
        S[2 * m + 1] = bf_hi(ws[m]);
        C[2 * m] = bf_lo(wc[m]);
        C[2 * m + 1] = bf_hi(wc[m]);
        N[2 * m] = bf_lo(wn[m]);
        N[2 * m + 1] = bf_hi(wn[m]);
      }
#pragma unroll
      for (int q = 0; q < 8; ++q)
        if (xc + q >= nx) S[q] = C[q] = N[q] = 0.f;  // columns of a straddling vector beyond the grid
      // west of lane 0's vector g is lane 31's vector g-1; east of lane 31's vector g is lane 0's vector g+1
      float wprev = 0.f, enext = 0.f;
      if (g > 0 && xs + 256 * (g - 1) + 8 * lane + 7 < nx) wprev = bf_hi(raw[k + 1][g - 1].w);
      if (g < G - 1 && xs + 256 * (g + 1) + 8 * lane < nx) enext = bf_lo(raw[k + 1][g + 1].x);
      const float wv = (lane == 31 && g > 0) ? wprev : C[7];
      const float ev = (lane == 0 && g < G - 1) ? enext : C[0];
      float left = __shfl_sync(0xffffffffu, wv, (lane + 31) & 31);
      float right = __shfl_sync(0xffffffffu, ev, (lane + 1) & 31);
      if (g == 0 && lane == 0) left = hl;
      if (g == G - 1 && lane == 31) right = hr;
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        const float w = q == 0 ? left : C[q - 1];
        const float e = q == 7 ? right : C[q + 1];
        float acc = 4.f * C[q];
        acc -= w;
        acc -= e;
        acc -= S[q];
        acc -= N[q];
        Y[q] = acc;
      }
      if (xc >= nx) continue;
      uint16_t* dst = y + (size_t)j * ld + xc;
      const uint4 o = make_uint4(bf_pack2(Y[0], Y[1]), bf_pack2(Y[2], Y[3]), bf_pack2(Y[4], Y[5]),
                                 bf_pack2(Y[6], Y[7]));
      if (xc + 8 <= nx) {
        *reinterpret_cast<uint4*>(dst) = o;
      } else {
        const uint32_t w[4] = {o.x, o.y, o.z, o.w};
#pragma unroll
        for (int q = 0; q < 8; ++q)
          if (xc + q < nx) dst[q] = (uint16_t)((q & 1) ? (w[q >> 1] >> 16) : (w[q >> 1] & 0xffffu));
      }
    }
  }
}

static int launch_apply_bf16x16(int nx, int ny, int ld, const void* x, void* y, cudaStream_t st) {
  const int ns = (nx + 256 * kBfGroups - 1) / (256 * kBfGroups);
  const long long blocks = (long long)ns * ((ny + kApplyWarps * kBfRows - 1) / (kApplyWarps * kBfRows));
  if (blocks > 0x7fffffffLL) return LAP5CG_ERR_INVALID_ARG;
  k_lap5_apply_bf16x16<<<(unsigned)blocks, 32 * kApplyWarps, 0, st>>>(nx, ny, ld, static_cast<const uint16_t*>(x),
                                                                       static_cast<uint16_t*>(y), ns);
  return cudaGetLastError() == cudaSuccess ? LAP5CG_OK : LAP5CG_ERR_CUDA;
}

template <class T, int V>
static int launch_apply(int nx, int ny, int ld, const void* x, void* y, cudaStream_t st) {
  constexpr int R = kApplyRows;
  const int ns = (nx + 32 * V - 1) / (32 * V);
  const long long blocks = (long long)ns * ((ny + kApplyWarps * R - 1) / (kApplyWarps * R));
  if (blocks > 0x7fffffffLL) return LAP5CG_ERR_INVALID_ARG;
  Grid<const T> gx{static_cast<const T*>(x), ld};
  Grid<T> gy{static_cast<T*>(y), ld};
  k_lap5_apply<T, V, R><<<(unsigned)blocks, 32 * kApplyWarps, 0, st>>>(nx, ny, gx, gy, ns);
  return cudaGetLastError() == cudaSuccess ? LAP5CG_OK : LAP5CG_ERR_CUDA;
}

static bool aligned(const void* p, size_t a) { return (reinterpret_cast<uintptr_t>(p) % a) == 0; }

// Vector widths: binary64 two columns a lane (FP64-bound: 4 operations a
// point), binary32 eight (two 16-byte groups 128 columns apart), bf16 sixteen
// (two 16-byte vectors; four where the pitch is a multiple of 4 only).
int apply_dispatch(int nx, int ny, int ld, int dtype, const void* x, void* y, cudaStream_t st) {
  switch (dtype) {
    case LAP5CG_DT_F64:
      if (ld % 2 == 0 && aligned(x, 16) && aligned(y, 16)) return launch_apply<double, 2>(nx, ny, ld, x, y, st);
      return launch_apply<double, 1>(nx, ny, ld, x, y, st);
    case LAP5CG_DT_F32:
      if (ld % 4 == 0 && aligned(x, 16) && aligned(y, 16)) return launch_apply<float, 8>(nx, ny, ld, x, y, st);
      return launch_apply<float, 1>(nx, ny, ld, x, y, st);
    case LAP5CG_DT_BF16:
      if (ld % 8 == 0 && aligned(x, 16) && aligned(y, 16)) return launch_apply_bf16x16(nx, ny, ld, x, y, st);
      if (ld % 4 == 0 && aligned(x, 8) && aligned(y, 8)) return launch_apply<bf16s, 4>(nx, ny, ld, x, y, st);
      return launch_apply<bf16s, 1>(nx, ny, ld, x, y, st);
    default:
      return LAP5CG_ERR_INVALID_ARG;
  }
}

}  // namespace lap5
