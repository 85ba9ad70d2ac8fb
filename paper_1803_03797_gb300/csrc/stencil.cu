// stencil.cu -- lap5_apply: y = A x for the 5-point Dirichlet Laplacian
// (arxiv 1803.03797, Sec. II-B mask), binary64 / binary32 / bf16 storage.
// One warp per (strip, row segment) unit, the same register line buffer as
// the solver passes; not persistent, no grid barrier.
#include "common.cuh"
#include "launch.h"

namespace lap5 {

template <class T, int V>
__global__ void __launch_bounds__(256) k_lap5_apply(int nx, int ny, Grid<const T> x, Grid<T> y, Units un) {
  using M = typename Math<T>::type;
  struct D { int dummy; };
  const int lane = threadIdx.x & 31;
  const int wpc = blockDim.x >> 5;
  const int gw = blockIdx.x * wpc + (threadIdx.x >> 5);
  const int nw = gridDim.x * wpc;
  for (int u = gw; u < un.nunits; u += nw) {
    int s, y0, y1;
    unit_bounds(un, u, ny, s, y0, y1);
    const int xs = s * 32 * V, xl = xs + lane * V;
    auto field = [&](int j, FRow<V, M>& f) {
      if (j < 0 || j >= ny) { f.zero(); return; }
      load_row<V>(x, j, xl, nx, f.f);
      f.hl = (lane == 0) ? load_one<const T, M>(x, j, xs - 1, nx) : M(0);
      f.hr = (lane == 31) ? load_one<const T, M>(x, j, xs + 32 * V, nx) : M(0);
    };
    auto load = [&](int, D&) {};
    auto finish = [&](int j, const D&, const FRow<V, M>& S, const FRow<V, M>& C, const FRow<V, M>& N) {
      M yv[V];
      stencil_row<V>(S, C, N, lane, yv);
      store_row<V>(y, j, xl, nx, yv);
    };
    march<V, M, D>(y0, y1, false, field, load, finish);
  }
}

template <class T, int V>
static int launch_apply(int nx, int ny, int ld, const void* x, void* y, cudaStream_t st) {
  Units un;
  un.ns = (nx + 32 * V - 1) / (32 * V);
  un.seg_rows = 32;
  un.nseg = (ny + un.seg_rows - 1) / un.seg_rows;
  un.nunits = un.ns * un.nseg;
  const int threads = 256, wpc = threads / 32;
  int blocks = (un.nunits + wpc - 1) / wpc;
  if (blocks > 65535) blocks = 65535;
  Grid<const T> gx{static_cast<const T*>(x), ld};
  Grid<T> gy{static_cast<T*>(y), ld};
  k_lap5_apply<T, V><<<blocks, threads, 0, st>>>(nx, ny, gx, gy, un);
  return cudaGetLastError() == cudaSuccess ? LAP5CG_OK : LAP5CG_ERR_CUDA;
}

static bool aligned(const void* p, size_t a) { return (reinterpret_cast<uintptr_t>(p) % a) == 0; }

int apply_dispatch(int nx, int ny, int ld, int dtype, const void* x, void* y, cudaStream_t st) {
  switch (dtype) {
    case LAP5CG_DT_F64:
      if (ld % 2 == 0 && aligned(x, 16) && aligned(y, 16)) return launch_apply<double, 2>(nx, ny, ld, x, y, st);
      return launch_apply<double, 1>(nx, ny, ld, x, y, st);
    case LAP5CG_DT_F32:
      if (ld % 4 == 0 && aligned(x, 16) && aligned(y, 16)) return launch_apply<float, 4>(nx, ny, ld, x, y, st);
      return launch_apply<float, 1>(nx, ny, ld, x, y, st);
    case LAP5CG_DT_BF16:
      if (ld % 4 == 0 && aligned(x, 8) && aligned(y, 8)) return launch_apply<bf16s, 4>(nx, ny, ld, x, y, st);
      return launch_apply<bf16s, 1>(nx, ny, ld, x, y, st);
    default:
      return LAP5CG_ERR_INVALID_ARG;
  }
}

}  // namespace lap5
