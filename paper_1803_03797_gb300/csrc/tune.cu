// tune.cu -- lap5cg_tune / lap5cg_tune_batched: pick launch parameters by
// timing real solves (CUDA events on the caller's stream).
//
// Search: coordinate descent from the given options.  Each round sweeps one
// parameter over its candidate values with the others fixed and keeps the
// fastest; two rounds over all parameters.  A trial is a fixed-iteration
// solve (tol = 0) from x = 0, so every trial does the same arithmetic.
#include <string.h>

#include "launch.h"

namespace lap5 {

struct Param {
  int32_t lap5cg_opts::*field;
  int values[6];
  int n;
};

static int time_trial(const lap5cg_opts& o, int (*run)(const lap5cg_opts&, void*), void* ctx, cudaStream_t st,
                      float* ms) {
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess) return LAP5CG_ERR_CUDA;
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return LAP5CG_ERR_CUDA;
  }
  int rc = run(o, ctx);  // warm-up (also validates the candidate)
  if (rc == LAP5CG_OK) {
    cudaEventRecord(e0, st);
    rc = run(o, ctx);
    cudaEventRecord(e1, st);
    if (rc == LAP5CG_OK && cudaEventSynchronize(e1) == cudaSuccess) {
      cudaEventElapsedTime(ms, e0, e1);
    } else if (rc == LAP5CG_OK) {
      rc = LAP5CG_ERR_CUDA;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return rc;
}

static int coordinate_descent(lap5cg_opts* o, const Param* params, int np, int (*run)(const lap5cg_opts&, void*),
                              void* ctx, cudaStream_t st, double* best_ms) {
  float best = 0.f;
  int rc = time_trial(*o, run, ctx, st, &best);
  if (rc != LAP5CG_OK) return rc;
  for (int round = 0; round < 2; ++round) {
    for (int p = 0; p < np; ++p) {
      lap5cg_opts cand = *o;
      for (int k = 0; k < params[p].n; ++k) {
        cand.*(params[p].field) = params[p].values[k];
        if (cand.*(params[p].field) == o->*(params[p].field)) continue;
        float ms = 0.f;
        if (time_trial(cand, run, ctx, st, &ms) != LAP5CG_OK) {
          cudaGetLastError();  // a candidate that does not fit is skipped
          continue;
        }
        if (ms < best) {
          best = ms;
          *o = cand;
        }
      }
    }
  }
  if (best_ms) *best_ms = best;
  return LAP5CG_OK;
}

struct SingleCtx {
  int nx, ny, ld, variant, precision, iters;
  const void* b;
  void* x;
  void* ws;
  size_t ws_bytes;
  lap5cg_info* info;
  cudaStream_t st;
  size_t es;
};

static int run_single(const lap5cg_opts& o, void* p) {
  SingleCtx* c = static_cast<SingleCtx*>(p);
  if (cudaMemset2DAsync(c->x, (size_t)c->ld * c->es, 0, (size_t)c->nx * c->es, c->ny, c->st) != cudaSuccess)
    return LAP5CG_ERR_CUDA;
  lap5cg_opts t = o;
  t.true_residual = 0;
  t.history = nullptr;
  return cg_solve(c->nx, c->ny, c->ld, c->b, c->x, 0.0, c->iters, c->variant, c->precision, 1, c->ws, c->ws_bytes,
                  c->info, &t, c->st);
}

struct BatchCtx {
  int count, variant, precision, iters;
  const int *nx, *ny, *ld;
  const void* const* b;
  void* const* x;
  void* ws;
  size_t ws_bytes;
  lap5cg_info* info;
  cudaStream_t st;
  size_t es;
};

static int run_batched(const lap5cg_opts& o, void* p) {
  BatchCtx* c = static_cast<BatchCtx*>(p);
  for (int k = 0; k < c->count; ++k)
    if (cudaMemset2DAsync(c->x[k], (size_t)c->ld[k] * c->es, 0, (size_t)c->nx[k] * c->es, c->ny[k], c->st) !=
        cudaSuccess)
      return LAP5CG_ERR_CUDA;
  lap5cg_opts t = o;
  t.true_residual = 0;
  t.history = nullptr;
  // iters > 0: every instance runs that many iterations; iters == 0: every
  // instance solves to a relative residual of 1e-4, so that the work per
  // instance grows with its size as in a real solve (the queue's tail then
  // weighs as it will)
  const double tol = c->iters > 0 ? 0.0 : 1e-4;
  const int maxit = c->iters > 0 ? c->iters : 10000000;
  return cg_solve_batched(c->count, c->nx, c->ny, c->ld, c->b, c->x, tol, maxit, c->variant, c->precision, c->ws,
                          c->ws_bytes, c->info, &t, c->st);
}

}  // namespace lap5

using namespace lap5;

extern "C" LAP5CG_API int lap5cg_tune(int nx, int ny, int ld, const void* b, void* x, int variant, int precision,
                                      int iters, void* workspace, size_t ws_bytes, lap5cg_info* info,
                                      lap5cg_opts* opts, double* best_ms, void* stream) {
  if (!opts || iters < 1 || !b || !x) return LAP5CG_ERR_INVALID_ARG;
  SingleCtx c{nx, ny, ld, variant, precision, iters, b, x, workspace, ws_bytes, info,
              static_cast<cudaStream_t>(stream), (size_t)(precision == LAP5CG_PREC_F32 ? 4 : 8)};
  Param params[5] = {{&lap5cg_opts::warps_per_cta, {4, 8, 16}, 3},
                     {&lap5cg_opts::ring_slots, {-1, 3, 4, 6, 8}, 5},
                     {&lap5cg_opts::min_rows, {4, 8, 16, 32, 64}, 5}};
  int np = 3;
  if (variant == LAP5CG_CLASSIC && precision != LAP5CG_PREC_IR_F32 && precision != LAP5CG_PREC_IR_BF16PR)
    params[np++] = {&lap5cg_opts::store_z, {0, 1}, 2};
  if (variant == LAP5CG_CLASSIC && precision != LAP5CG_PREC_F64)  // binary32 passes: lane vector width
    params[np++] = {&lap5cg_opts::lane_vec, {4, 8}, 2};
  else if (variant == LAP5CG_CLASSIC)  // binary64 classic: two or four columns a lane
    params[np++] = {&lap5cg_opts::lane_vec, {2, 4}, 2};
  return coordinate_descent(opts, params, np, run_single, &c, c.st, best_ms);
}

extern "C" LAP5CG_API int lap5cg_tune_batched(int count, const int* nx, const int* ny, const int* ld,
                                              const void* const* b, void* const* x, int variant, int precision,
                                              int iters, void* workspace, size_t ws_bytes, lap5cg_info* info,
                                              lap5cg_opts* opts, double* best_ms, void* stream) {
  if (!opts || iters < 0 || count < 1 || !nx || !ny || !ld || !b || !x) return LAP5CG_ERR_INVALID_ARG;
  BatchCtx c{count, variant, precision, iters, nx, ny, ld, b, x, workspace, ws_bytes, info,
             static_cast<cudaStream_t>(stream), (size_t)(precision == LAP5CG_PREC_F32 ? 4 : 8)};
  Param params[4] = {{&lap5cg_opts::team_ctas, {1, 2, 4, 8, 16}, 5},
                     {&lap5cg_opts::warps_per_cta, {4, 8, 16}, 3},
                     {&lap5cg_opts::ring_slots, {-1, 3, 4, 6}, 4},
                     {&lap5cg_opts::min_rows, {4, 8, 16, 32}, 4}};
  return coordinate_descent(opts, params, 4, run_batched, &c, c.st, best_ms);
}
