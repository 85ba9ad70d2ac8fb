// probe.cu -- lap5cg_fp64_rate: the FP64 fused multiply-add and add rates of
// the current GPU, measured with a throughput kernel.  The binary64 solver
// kernels are bound by the FP64 pipe rather than by memory, so the benchmark
// reports them against this measured rate instead of a nominal one.
#include "launch.h"

namespace lap5 {

constexpr int kProbeChains = 8;     // independent dependency chains a thread
constexpr int kProbeThreads = 256;
constexpr int kProbeBlocksPerSm = 8;  // 64 warps an SM

// Written only if the chains reach an impossible value: keeps them live
// without a caller buffer.
static __device__ double g_probe_sink;

template <bool FMA>
__global__ void __launch_bounds__(kProbeThreads) k_fp64_rate(int iters, double seed) {
  double a[kProbeChains];
#pragma unroll
  for (int k = 0; k < kProbeChains; ++k) a[k] = seed + (double)k + 1e-9 * threadIdx.x;
  // multiplier and addend in registers (per-thread values), not constant operands
  const double m = 1.0 - 1e-12 * (double)(1 + (threadIdx.x & 1)), c = 1e-13 * (double)(1 + (threadIdx.x & 2));
#pragma unroll 4
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < kProbeChains; ++k) a[k] = FMA ? __fma_rn(a[k], m, c) : __dadd_rn(a[k], c);
  }
  double s = 0.0;
#pragma unroll
  for (int k = 0; k < kProbeChains; ++k) s += a[k];
  if (s == -1.0) g_probe_sink = s;  // the chains stay near seed + k > 0
}

template <bool FMA>
static int time_rate(int blocks, int iters, cudaStream_t st, cudaEvent_t e0, cudaEvent_t e1, double* per_s) {
  k_fp64_rate<FMA><<<blocks, kProbeThreads, 0, st>>>(iters / 8, 1.0);  // warm-up
  double best = 0.0;
  for (int rep = 0; rep < 5; ++rep) {
    if (cudaEventRecord(e0, st) != cudaSuccess) return LAP5CG_ERR_CUDA;
    k_fp64_rate<FMA><<<blocks, kProbeThreads, 0, st>>>(iters, 1.0);
    if (cudaGetLastError() != cudaSuccess || cudaEventRecord(e1, st) != cudaSuccess ||
        cudaEventSynchronize(e1) != cudaSuccess)
      return LAP5CG_ERR_CUDA;
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess || ms <= 0.f) return LAP5CG_ERR_CUDA;
    const double ops = (double)blocks * kProbeThreads * kProbeChains * (double)iters;
    const double r = ops / (ms * 1e-3);
    if (r > best) best = r;
  }
  *per_s = best;
  return LAP5CG_OK;
}

}  // namespace lap5

using namespace lap5;

extern "C" LAP5CG_API int lap5cg_fp64_rate(double* fma_per_s, double* add_per_s, void* stream) {
  if (!fma_per_s || !add_per_s) return LAP5CG_ERR_INVALID_ARG;
  DevProps dp;
  int rc = dev_props(&dp);
  if (rc != LAP5CG_OK) return rc;
  const int blocks = dp.sms * kProbeBlocksPerSm;
  const int iters = 10000;  // about 40 ms a launch on a GB300
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess) return LAP5CG_ERR_CUDA;
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return LAP5CG_ERR_CUDA;
  }
  rc = time_rate<true>(blocks, iters, st, e0, e1, fma_per_s);
  if (rc == LAP5CG_OK) rc = time_rate<false>(blocks, iters, st, e0, e1, add_per_s);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return rc;
}
