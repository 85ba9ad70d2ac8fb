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
#include <cuda.h>
#include <cudaTypedefs.h>

#include <atomic>
#include <mutex>

#include "common.cuh"
#include "launch.h"
#include "ring.cuh"

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

// bf16 storage through TMA tiles.  A tile is 16 output rows of 256 columns;
// its operand rows (18 of 256 columns) and the one-column halos left and right
// (two 8-column boxes, the narrowest 16-byte box) land in shared memory by
// three tensor copies.  The tensor map spans exactly nx x ny, so every operand
// outside the grid -- the Dirichlet boundary, the ragged right and bottom
// edges -- arrives as the copy's zero fill, and no load is masked.  Persistent
// CTAs walk the tiles with three stages in flight; each thread finishes one
// 8-column vector in each of kTmaRowsPerThread rows with the arithmetic of the
// register kernel above, so the results are bit-identical.
constexpr int kTmaW = 256, kTmaH = 16, kTmaStages = 3, kTmaThreads = 256;
constexpr int kTmaRowsPerThread = kTmaH / (kTmaThreads / 32);
static_assert(kTmaH % (kTmaThreads / 32) == 0, "whole rows a warp");
constexpr int kTmaMainBytes = kTmaW * (kTmaH + 2) * 2;                // 9216
constexpr int kTmaHaloBytes = 8 * (kTmaH + 2) * 2;                    // 288
constexpr int kTmaHaloStride = (kTmaHaloBytes + 127) / 128 * 128;     // 128-byte aligned slots
static_assert(kTmaMainBytes % 128 == 0 && kTmaHaloStride >= kTmaHaloBytes, "stage layout");
static_assert(kTmaH + 2 <= 256 && kTmaW <= 256, "tensor-copy box extents");
constexpr int kTmaStageBytes = kTmaMainBytes + 2 * kTmaHaloStride;
constexpr uint32_t kTmaTx = kTmaMainBytes + 2 * kTmaHaloBytes;

// Diagnostics: stages whose copy did not land within the wait limit, plus
// 65536 for each CTA that found its shared memory misaligned for the copies
// (and wrote nothing).
__device__ int g_apply_tma_timeouts;

__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap* map, int x, int y, uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
          dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(bar)
      : "memory");
}

// Bounded wait on a stage's barrier; false when it ran out (the copy is
// waited for once more, also bounded, so that none is in flight at exit).
__device__ __forceinline__ bool tma_wait(uint32_t bar, uint32_t parity) {
  for (int round = 0; round < 2; ++round) {
    const unsigned long long t0 = global_ns();
    unsigned spins = 0;
    for (;;) {
      uint32_t ok;
      asm volatile(
          "{\n\t.reg .pred p;\n\t"
          "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
          "selp.u32 %0, 1, 0, p;\n\t}"
          : "=r"(ok)
          : "r"(bar), "r"(parity), "r"(kSuspendHintNs)
          : "memory");
      if (ok) return round == 0;
      if ((++spins & 63u) == 0u && global_ns() - t0 > 1000000000ull) break;
    }
    if (round == 0 && threadIdx.x == 0) atomicAdd(&g_apply_tma_timeouts, 1);
  }
  return false;
}

__global__ void __launch_bounds__(kTmaThreads) k_lap5_apply_bf16_tma(const __grid_constant__ CUtensorMap mmain,
                                                                    const __grid_constant__ CUtensorMap mhalo,
                                                                    int nx, int ny, int ld, uint16_t* __restrict__ y,
                                                                    int tiles_x, int ntiles) {
  // stages first, then the barriers; no static shared memory, so the stages
  // start at the (aligned) beginning of the dynamic window
  extern __shared__ __align__(128) unsigned char tsm[];
  const uint32_t base = smem_u32(tsm), bar0 = base + (uint32_t)(kTmaStages * kTmaStageBytes);
  if (base & 127u) {  // tensor copies need 128-byte aligned destinations
    if (threadIdx.x == 0) atomicAdd(&g_apply_tma_timeouts, 1 << 16);
    return;
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (threadIdx.x == 0) {
    for (int sidx = 0; sidx < kTmaStages; ++sidx)
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar0 + 8u * sidx) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  auto issue = [&](int t, int sidx) {  // thread 0
    const int x0 = (t % tiles_x) * kTmaW, y0 = (t / tiles_x) * kTmaH;
    const uint32_t bar = bar0 + 8u * sidx, dst = base + (uint32_t)(sidx * kTmaStageBytes);
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(kTmaTx) : "memory");
    tma_load_2d(dst, &mmain, x0, y0 - 1, bar);
    tma_load_2d(dst + kTmaMainBytes, &mhalo, x0 - 8, y0 - 1, bar);
    tma_load_2d(dst + kTmaMainBytes + kTmaHaloStride, &mhalo, x0 + kTmaW, y0 - 1, bar);
  };
  const int first = blockIdx.x, step = gridDim.x;
  if (threadIdx.x == 0)
    for (int k = 0; k < kTmaStages; ++k)
      if (first + k * step < ntiles) issue(first + k * step, k);
  bool ok = true;
  int k = 0;
  for (int t = first; t < ntiles; t += step, ++k) {
    const int sidx = k % kTmaStages;
    ok = tma_wait(bar0 + 8u * sidx, (uint32_t)((k / kTmaStages) & 1)) && ok;
    const unsigned char* st = tsm + sidx * kTmaStageBytes;
    const uint16_t* mrow = reinterpret_cast<const uint16_t*>(st);
    const uint16_t* hl = reinterpret_cast<const uint16_t*>(st + kTmaMainBytes);
    const uint16_t* hr = reinterpret_cast<const uint16_t*>(st + kTmaMainBytes + kTmaHaloStride);
    const int x0 = (t % tiles_x) * kTmaW, y0 = (t / tiles_x) * kTmaH;
    const int xc = x0 + 8 * lane;
#pragma unroll
    for (int h = 0; h < kTmaRowsPerThread; ++h) {
      const int r = warp + (kTmaThreads / 32) * h;  // output row y0 + r; operand rows r .. r + 2 of the stage
      const uint4 rs = *reinterpret_cast<const uint4*>(mrow + r * kTmaW + 8 * lane);
      const uint4 rc = *reinterpret_cast<const uint4*>(mrow + (r + 1) * kTmaW + 8 * lane);
      const uint4 rn = *reinterpret_cast<const uint4*>(mrow + (r + 2) * kTmaW + 8 * lane);
      const uint32_t ws[4] = {rs.x, rs.y, rs.z, rs.w}, wc[4] = {rc.x, rc.y, rc.z, rc.w},
                     wn[4] = {rn.x, rn.y, rn.z, rn.w};
      float S[8], C[8], N[8], Y[8];
#pragma unroll
      for (int m = 0; m < 4; ++m) {
        S[2 * m] = bf_lo(ws[m]);
        S[2 * m + 1] = bf_hi(ws[m]);
        C[2 * m] = bf_lo(wc[m]);
        C[2 * m + 1] = bf_hi(wc[m]);
        N[2 * m] = bf_lo(wn[m]);
        N[2 * m + 1] = bf_hi(wn[m]);
      }
      float left = __shfl_sync(0xffffffffu, C[7], (lane + 31) & 31);
      float right = __shfl_sync(0xffffffffu, C[0], (lane + 1) & 31);
      if (lane == 0) left = bf_widen(hl[(r + 1) * 8 + 7]);
      if (lane == 31) right = bf_widen(hr[(r + 1) * 8]);
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
      const int j = y0 + r;
      if (!ok || j >= ny || xc >= nx) continue;
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
    __syncthreads();  // every thread is done with this stage
    if (threadIdx.x == 0 && t + kTmaStages * step < ntiles) {
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      issue(t + kTmaStages * step, sidx);
    }
  }
}

static PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  });
  return fn;
}

// LAP5CG_ERR_UNSUPPORTED when the tensor maps cannot be made (the caller
// takes the register kernel).
static int launch_apply_bf16_tma(int nx, int ny, int ld, const void* x, void* y, cudaStream_t st) {
  const PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
  if (!enc) return LAP5CG_ERR_UNSUPPORTED;
  CUtensorMap mmain, mhalo;
  const cuuint64_t dims[2] = {(cuuint64_t)nx, (cuuint64_t)ny};
  const cuuint64_t strides[1] = {(cuuint64_t)ld * 2};
  const cuuint32_t box_main[2] = {(cuuint32_t)kTmaW, (cuuint32_t)(kTmaH + 2)};
  const cuuint32_t box_halo[2] = {8u, (cuuint32_t)(kTmaH + 2)};
  const cuuint32_t estr[2] = {1u, 1u};
  void* gx = const_cast<void*>(x);
  if (enc(&mmain, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, gx, dims, strides, box_main, estr,
          CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
          CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS ||
      enc(&mhalo, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, gx, dims, strides, box_halo, estr,
          CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
          CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
    return LAP5CG_ERR_UNSUPPORTED;
  const int tiles_x = (nx + kTmaW - 1) / kTmaW;
  const long long nt = (long long)tiles_x * ((ny + kTmaH - 1) / kTmaH);
  if (nt > 0x7fffffffLL) return LAP5CG_ERR_UNSUPPORTED;
  const size_t smem = (size_t)kTmaStages * kTmaStageBytes + 8 * kTmaStages;
  DevProps dp;
  const int rc = dev_props(&dp);
  if (rc != LAP5CG_OK) return rc;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 128) return LAP5CG_ERR_CUDA;
  // The shared-memory size attribute, set once per device (its host cost would
  // show in front of a kernel of tens of microseconds), and set again with the
  // launch retried once if a launch is refused (a device reset drops it).
  static std::atomic<int> attr_set[128];
  auto set_attr = [&]() {
    return cudaFuncSetAttribute(k_lap5_apply_bf16_tma, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) ==
           cudaSuccess;
  };
  if (!attr_set[dev].load(std::memory_order_relaxed)) {
    if (!set_attr()) return LAP5CG_ERR_CUDA;
    attr_set[dev].store(1, std::memory_order_relaxed);
  }
  // resident CTAs an SM, per device (the occupancy query costs microseconds of
  // host time as well)
  static std::atomic<int> occ_cache[128];
  int occ = occ_cache[dev].load(std::memory_order_relaxed);
  if (occ == 0) {
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_lap5_apply_bf16_tma, kTmaThreads, smem) != cudaSuccess ||
        occ < 1)
      occ = 1;
    occ_cache[dev].store(occ, std::memory_order_relaxed);
  }
  const long long grid = std::min<long long>(nt, (long long)occ * dp.sms);
  auto launch = [&]() {
    k_lap5_apply_bf16_tma<<<(unsigned)grid, kTmaThreads, smem, st>>>(mmain, mhalo, nx, ny, ld,
                                                                    static_cast<uint16_t*>(y), tiles_x, (int)nt);
    return cudaGetLastError();
  };
  cudaError_t e = launch();
  if (e != cudaSuccess && set_attr()) e = launch();
  return e == cudaSuccess ? LAP5CG_OK : LAP5CG_ERR_CUDA;
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
      if (ld % 8 == 0 && aligned(x, 16) && aligned(y, 16)) {
        const int rc = launch_apply_bf16_tma(nx, ny, ld, x, y, st);
        if (rc != LAP5CG_ERR_UNSUPPORTED) return rc;
        return launch_apply_bf16x16(nx, ny, ld, x, y, st);
      }
      if (ld % 4 == 0 && aligned(x, 8) && aligned(y, 8)) return launch_apply<bf16s, 4>(nx, ny, ld, x, y, st);
      return launch_apply<bf16s, 1>(nx, ny, ld, x, y, st);
    default:
      return LAP5CG_ERR_INVALID_ARG;
  }
}

}  // namespace lap5
