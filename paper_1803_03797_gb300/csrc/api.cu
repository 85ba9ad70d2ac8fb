// api.cu -- the extern "C" entry points of liblap5cg (declared in
// include/lap5cg.h): argument validation, workspace layout, staging of
// unaligned user buffers, launch-geometry planning and dispatch.
#include <mutex>
#include <string.h>

#include "launch.h"
#include "common.cuh"

namespace lap5 {

int dev_props(DevProps* out) {
  static std::mutex mu;
  static DevProps cache[128];
  static bool have[128] = {false};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 128) return LAP5CG_ERR_CUDA;
  std::lock_guard<std::mutex> lock(mu);
  if (!have[dev]) {
    DevProps p;
    if (cudaDeviceGetAttribute(&p.sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return LAP5CG_ERR_CUDA;
    if (cudaDeviceGetAttribute(&p.max_smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess)
      return LAP5CG_ERR_CUDA;
    cache[dev] = p;
    have[dev] = true;
  }
  *out = cache[dev];
  return LAP5CG_OK;
}

int warps_of(const lap5cg_opts& o) {
  int wpc = o.warps_per_cta > 0 ? o.warps_per_cta : kDefaultWarps;
  return wpc > 16 ? 16 : wpc;
}

int plan_units(const void* func, int nx, int ny, int V, const lap5cg_opts& o, size_t dyn_smem, LaunchCfg* cfg,
               int row_align) {
  DevProps dp;
  int rc = dev_props(&dp);
  if (rc != LAP5CG_OK) return rc;
  const int wpc = warps_of(o);
  const int threads = 32 * wpc;
  int occ = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, func, threads, dyn_smem) != cudaSuccess)
    return LAP5CG_ERR_CUDA;
  if (occ < 1) return LAP5CG_ERR_UNSUPPORTED;
  int maxctas = occ * dp.sms;
  if (maxctas > kMaxCtas) maxctas = kMaxCtas;
  int ctas = o.ctas > 0 ? (o.ctas < maxctas ? o.ctas : maxctas) : maxctas;
  const long long W = (long long)ctas * wpc;
  const Units un = make_units(nx, ny, V, W, o.min_rows > 0 ? o.min_rows : kDefaultMinRows, row_align);
  const long long nunits = un.nunits;
  if (o.ctas <= 0 && nunits < W) ctas = (int)((nunits + wpc - 1) / wpc);
  cfg->ctas = ctas;
  cfg->threads = threads;
  cfg->dyn_smem = dyn_smem;
  cfg->ns = un.ns;
  cfg->nseg = un.nseg;
  cfg->seg_rows = un.seg_rows;
  cfg->nunits = un.nunits;
  return LAP5CG_OK;
}

int choose_ring(const void* func, int slot_bytes, const lap5cg_opts& o, int wpc, RingGeom* g, size_t* dyn_smem,
                bool auto_on) {
  g->S = 0;
  g->slot_bytes = slot_bytes;
  g->warp_bytes = 0;
  *dyn_smem = 0;
  if (o.ring_slots < 0 || (o.ring_slots == 0 && !auto_on)) return LAP5CG_OK;
  if (wpc < 1 || wpc > 16) return LAP5CG_ERR_INVALID_ARG;
  const int budget = wpc * kRingBytesPerWarp;
  int S;
  if (o.ring_slots > 0) {
    S = o.ring_slots < 3 ? 3 : (o.ring_slots > kRingMaxSlots ? kRingMaxSlots : o.ring_slots);
  } else {
    S = (budget / wpc - 128) / slot_bytes;
    if (S > 6) S = 6;
    if (S < 3) return LAP5CG_OK;  // too little room: register march
  }
  const int warp_bytes = (int)align_up(128 + (size_t)S * slot_bytes, 128);
  const size_t dyn = (size_t)wpc * warp_bytes;
  DevProps dp;
  int rc = dev_props(&dp);
  if (rc != LAP5CG_OK) return rc;
  if (dyn > (size_t)dp.max_smem_optin) {
    if (o.ring_slots > 0) return LAP5CG_ERR_UNSUPPORTED;
    return LAP5CG_OK;
  }
  if (cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn) != cudaSuccess)
    return LAP5CG_ERR_CUDA;
  g->S = S;
  g->warp_bytes = warp_bytes;
  *dyn_smem = dyn;
  return LAP5CG_OK;
}

static bool aligned(const void* p, size_t a) { return (reinterpret_cast<uintptr_t>(p) % a) == 0; }

static size_t elem_of_precision(int precision) { return precision == LAP5CG_PREC_F32 ? 4 : 8; }

// Lane vector width of the solver kernels for a precision: binary64 2,
// binary32 4, mixed-precision kernels 4 (binary64 b and x read 32 bytes a lane).
// Pitch granule (elements) of the arrays a solve reads with vector loads.  The
// multigrid solve reads its binary64 r four columns a lane in the V-cycle's
// binary32 layout, so its internal pitch is a multiple of 4 as well.
static int vec_of_precision(int precision) { return precision == LAP5CG_PREC_F64 ? 2 : 4; }

static int internal_ld(int nx, int ld, int precision) {
  const int v = vec_of_precision(precision);
  if (ld % v == 0) return ld;
  return (nx + v - 1) / v * v;
}

static size_t solver_ws(int nx, int ny, int ldw, int variant, int precision) {
  switch (precision) {
    case LAP5CG_PREC_F64: return ws_bytes_f64(nx, ny, ldw, variant);
    case LAP5CG_PREC_F32: return ws_bytes_f32(nx, ny, ldw, variant);
    case LAP5CG_PREC_MG_F32:
    case LAP5CG_PREC_MG_F64: return ws_bytes_mg(nx, ny, ldw, variant, precision);
    default: return ws_bytes_ir(nx, ny, variant, precision);
  }
}

static bool valid_shape(int nx, int ny, int ld) {
  if (nx < 1 || ny < 1 || ld < nx) return false;
  if ((long long)ny * (long long)ld > (1LL << 40)) return false;
  return true;
}

static bool overlap(const void* a, size_t na, const void* b, size_t nb) {
  const uintptr_t a0 = reinterpret_cast<uintptr_t>(a), b0 = reinterpret_cast<uintptr_t>(b);
  return a0 < b0 + nb && b0 < a0 + na;
}

}  // namespace lap5

using namespace lap5;

extern "C" {

void lap5cg_opts_default(lap5cg_opts* o) {
  if (!o) return;
  memset(o, 0, sizeof(*o));
  o->rr_period = 0;
  o->store_z = -1;
  o->ctas = 0;
  o->warps_per_cta = 0;
  o->min_rows = 0;
  o->true_residual = 1;
  o->maxit_inner = 0;
  o->max_outer = 0;
  o->tol_inner = 0.0;
  o->timeout_s = 0.0;
  o->history = nullptr;
  o->team_ctas = 0;
  o->ring_slots = 0;
  o->resident = 0;
  o->lane_vec = 0;
  o->reproducible = 0;
  o->mg_nu = 0;
  o->mg_levels = 0;
  o->mg_coarse_sweeps = 0;
  o->stabilized = 0;
}

const char* lap5cg_status_string(int status) {
  switch (status) {
    case LAP5CG_OK: return "ok";
    case LAP5CG_NOT_CONVERGED: return "not converged (maxit reached)";
    case LAP5CG_ERR_INVALID_ARG: return "invalid argument";
    case LAP5CG_ERR_CUDA: return "CUDA runtime error";
    case LAP5CG_ERR_BREAKDOWN: return "breakdown: non-positive curvature or alpha denominator";
    case LAP5CG_ERR_SYNC_TIMEOUT: return "device grid barrier timed out";
    case LAP5CG_ERR_NONFINITE: return "non-finite value in a reduction";
    case LAP5CG_ERR_UNSUPPORTED: return "unsupported combination";
    case LAP5CG_ERR_WORKSPACE: return "workspace missing, misaligned or too small";
    default: return "unknown status";
  }
}

int lap5_apply(int nx, int ny, int ld, int dtype, const void* x, void* y, void* stream) {
  if (!valid_shape(nx, ny, ld) || !x || !y) return LAP5CG_ERR_INVALID_ARG;
  if (dtype < LAP5CG_DT_F64 || dtype > LAP5CG_DT_BF16) return LAP5CG_ERR_INVALID_ARG;
  const size_t es = dtype == LAP5CG_DT_F64 ? 8 : (dtype == LAP5CG_DT_F32 ? 4 : 2);
  const size_t bytes = (size_t)ny * (size_t)ld * es;
  if (overlap(x, bytes, y, bytes)) return LAP5CG_ERR_INVALID_ARG;
  return apply_dispatch(nx, ny, ld, dtype, x, y, static_cast<cudaStream_t>(stream));
}

size_t cg_workspace_size(int nx, int ny, int ld, int variant, int precision, int nrhs) {
  if (!valid_shape(nx, ny, ld) || nrhs < 1) return 0;
  if (variant != LAP5CG_CLASSIC && variant != LAP5CG_NEWCG) return 0;
  if (precision < LAP5CG_PREC_F64 || precision > LAP5CG_PREC_MG_F64) return 0;
  const int ldw = internal_ld(nx, ld, precision);
  size_t s = solver_ws(nx, ny, ldw, variant, precision);
  if (s == 0) return 0;
  if (ldw != ld) s += 2 * align_up((size_t)ny * (size_t)ldw * elem_of_precision(precision), kAlign);
  return s;
}

int cg_solve(int nx, int ny, int ld, const void* b, void* x, double tol, int maxit, int variant, int precision,
             int nrhs, void* workspace, size_t ws_bytes, lap5cg_info* info, const lap5cg_opts* opts,
             void* stream) {
  if (!valid_shape(nx, ny, ld) || !b || !x || !info || maxit < 0 || nrhs < 1) return LAP5CG_ERR_INVALID_ARG;
  if (variant != LAP5CG_CLASSIC && variant != LAP5CG_NEWCG) return LAP5CG_ERR_INVALID_ARG;
  if (precision < LAP5CG_PREC_F64 || precision > LAP5CG_PREC_MG_F64) return LAP5CG_ERR_INVALID_ARG;
  if (tol != tol) return LAP5CG_ERR_INVALID_ARG;  // NaN tolerance
  lap5cg_opts o;
  if (opts) o = *opts;
  else lap5cg_opts_default(&o);
  if (o.rr_period < 0 || o.warps_per_cta < 0 || o.warps_per_cta > 16 || o.ctas < 0 || o.min_rows < 0 ||
      o.maxit_inner < 0 || o.max_outer < 0 || o.ring_slots > kRingMaxSlots || o.mg_nu < 0 || o.mg_levels < 0 ||
      o.mg_coarse_sweeps < 0 ||
      (o.lane_vec != 0 && o.lane_vec != 2 && o.lane_vec != 4 && o.lane_vec != 8) || o.reproducible < 0 || o.reproducible > 1)
    return LAP5CG_ERR_INVALID_ARG;
  if (o.reproducible && precision != LAP5CG_PREC_F64) return LAP5CG_ERR_UNSUPPORTED;
  if (o.reproducible && (long long)nx * (long long)ny >= (1ll << 36)) return LAP5CG_ERR_UNSUPPORTED;  // limb range
  if (o.rr_period > 0 && variant != LAP5CG_NEWCG) return LAP5CG_ERR_INVALID_ARG;
  if (o.stabilized < 0 || o.stabilized > 1 || (o.stabilized && variant != LAP5CG_NEWCG)) return LAP5CG_ERR_INVALID_ARG;
  if (o.stabilized && (o.reproducible || (precision != LAP5CG_PREC_F64 && precision != LAP5CG_PREC_F32)))
    return LAP5CG_ERR_UNSUPPORTED;
  const size_t need = cg_workspace_size(nx, ny, ld, variant, precision, nrhs);
  if (need == 0) return LAP5CG_ERR_UNSUPPORTED;
  if (!workspace || !aligned(workspace, kAlign) || ws_bytes < need) return LAP5CG_ERR_WORKSPACE;
  const size_t es = elem_of_precision(precision);
  const size_t grid_bytes = (size_t)ny * (size_t)ld * es;
  if (overlap(b, grid_bytes * nrhs, x, grid_bytes * nrhs)) return LAP5CG_ERR_INVALID_ARG;
  if (overlap(b, grid_bytes * nrhs, workspace, ws_bytes) || overlap(x, grid_bytes * nrhs, workspace, ws_bytes))
    return LAP5CG_ERR_INVALID_ARG;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const int ldw = internal_ld(nx, ld, precision);
  const bool vec_ok = (ldw == ld) && aligned(b, 16) && aligned(x, 16);
  const bool stage = !vec_ok;
  if (stage && ldw == ld) return LAP5CG_ERR_INVALID_ARG;  // aligned pitch but misaligned pointers
  unsigned char* ws = static_cast<unsigned char*>(workspace);
  const size_t solver_bytes = solver_ws(nx, ny, ldw, variant, precision);
  const size_t stage_vec = align_up((size_t)ny * (size_t)ldw * es, kAlign);
  unsigned char* bst = ws + solver_bytes;
  unsigned char* xst = bst + stage_vec;

  for (int k = 0; k < nrhs; ++k) {
    const unsigned char* bk = static_cast<const unsigned char*>(b) + (size_t)k * grid_bytes;
    unsigned char* xk = static_cast<unsigned char*>(x) + (size_t)k * grid_bytes;
    SolvePlan p;
    p.nx = nx;
    p.ny = ny;
    p.ldw = ldw;
    p.ws = ws;
    p.ws_bytes = solver_bytes;
    p.info = info + k;
    p.tol = tol;
    p.maxit = maxit;
    p.variant = variant;
    p.precision = precision;
    p.opts = o;
    if (o.history) p.opts.history = o.history + (size_t)k * ((size_t)maxit + 1);
    if (stage) {
      if (cudaMemcpy2DAsync(bst, (size_t)ldw * es, bk, (size_t)ld * es, (size_t)nx * es, ny, cudaMemcpyDeviceToDevice,
                            st) != cudaSuccess ||
          cudaMemcpy2DAsync(xst, (size_t)ldw * es, xk, (size_t)ld * es, (size_t)nx * es, ny, cudaMemcpyDeviceToDevice,
                            st) != cudaSuccess)
        return LAP5CG_ERR_CUDA;
      p.b = bst;
      p.x = xst;
      p.ld = ldw;
    } else {
      p.b = bk;
      p.x = xk;
      p.ld = ld;
    }
    int rc;
    bool done = false;
    rc = try_small(p, st, &done);  // small grids: one cluster, shared-memory resident
    if (rc != LAP5CG_OK) return rc;
    if (!done) {
      switch (precision) {
        case LAP5CG_PREC_F64: rc = solve_f64(p, st); break;
        case LAP5CG_PREC_F32: rc = solve_f32(p, st); break;
        case LAP5CG_PREC_MG_F32:
        case LAP5CG_PREC_MG_F64: rc = solve_mg(p, st); break;
        default: rc = solve_ir(p, st); break;
      }
    }
    if (rc != LAP5CG_OK) return rc;
    if (stage) {
      if (cudaMemcpy2DAsync(xk, (size_t)ld * es, xst, (size_t)ldw * es, (size_t)nx * es, ny, cudaMemcpyDeviceToDevice,
                            st) != cudaSuccess)
        return LAP5CG_ERR_CUDA;
    }
  }
  return LAP5CG_OK;
}

size_t cg_batched_workspace_size(int count, const int* nx, const int* ny, const int* ld, int variant,
                                 int precision) {
  if (variant != LAP5CG_CLASSIC && variant != LAP5CG_NEWCG) return 0;
  return batched_ws(count, nx, ny, ld, variant, precision);
}

int cg_solve_batched(int count, const int* nx, const int* ny, const int* ld, const void* const* b, void* const* x,
                     double tol, int maxit, int variant, int precision, void* workspace, size_t ws_bytes,
                     lap5cg_info* info, const lap5cg_opts* opts, void* stream) {
  if (count < 1 || count > LAP5CG_MAX_BATCH || !nx || !ny || !ld || !b || !x || !info || maxit < 0)
    return LAP5CG_ERR_INVALID_ARG;
  if (variant != LAP5CG_CLASSIC && variant != LAP5CG_NEWCG) return LAP5CG_ERR_INVALID_ARG;
  if (precision < LAP5CG_PREC_F64 || precision > LAP5CG_PREC_IR_BF16PR) return LAP5CG_ERR_INVALID_ARG;
  if (tol != tol) return LAP5CG_ERR_INVALID_ARG;
  lap5cg_opts o;
  if (opts) o = *opts;
  else lap5cg_opts_default(&o);
  if (o.rr_period < 0 || o.warps_per_cta < 0 || o.warps_per_cta > 16 || o.ctas < 0 || o.min_rows < 0 ||
      o.maxit_inner < 0 || o.max_outer < 0 || o.team_ctas < 0)
    return LAP5CG_ERR_INVALID_ARG;
  if (o.rr_period > 0 && variant != LAP5CG_NEWCG) return LAP5CG_ERR_INVALID_ARG;
  if (o.reproducible) return LAP5CG_ERR_UNSUPPORTED;  // exact dot products: single solves only
  if (o.stabilized) return LAP5CG_ERR_UNSUPPORTED;    // single solves only
  return solve_batched(count, nx, ny, ld, b, x, tol, maxit, variant, precision, workspace, ws_bytes, info, o,
                       static_cast<cudaStream_t>(stream));
}

}  // extern "C"
