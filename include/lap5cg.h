/*
 * lap5cg.h -- C ABI of liblap5cg: matrix-free conjugate gradient for the 2D
 * Dirichlet 5-point Laplacian on an NVIDIA GB300 (sm_103a).
 *
 * Method: arxiv 1803.03797, "Efficient FPGA Implementation of Conjugate
 * Gradient Methods for Laplacian System using HLS".
 *   - Problem (Sec. II): solve A x = b on an nx-by-ny interior grid of the unit
 *     square with zero Dirichlet boundary.  A is the 5-point stencil with the
 *     3x3 mask [0 -1 0; -1 4 -1; 0 -1 0] printed in Sec. II-B (symmetric
 *     positive definite, no 1/h^2 scaling), applied matrix-free.
 *   - Classic CG: Algorithm 1 (stdCG).
 *   - NewCG: Algorithm 2, the pipelined CG of Ghysels & Vanroose (M = I) that
 *     lets the stencil overlap the two dot products (Sec. II, Fig. NewCG).
 *
 * Data layout (all entry points): a grid is ny rows of ld elements (ld >= nx,
 * the row pitch in elements); element (i, j), 0 <= i < nx, 0 <= j < ny, is at
 * offset j*ld + i.  A buffer holds ny*ld elements.  Padding columns
 * nx <= i < ld are never written.  Boundary values are implicit zeros and are
 * not stored.
 *
 * Ownership: the caller owns every buffer (inputs, outputs, workspace, info).
 * No entry point below allocates device memory at call time, and the library
 * keeps no mutable global state apart from a per-device cache of device
 * properties (with the bf16 lap5_apply kernel's occupancy and whether its
 * shared-memory size is set; a refused launch sets it again) and, for the
 * classic multigrid-preconditioned solve (MG_F32, MG_F64), a cache of up to
 * eight instantiated CUDA graphs keyed by device, shape, workspace address and
 * V-cycle options: the first solve of a key builds and instantiates its graph
 * (driver-side resources, freed when the entry is evicted or by
 * lap5cg_release_graphs), later ones launch it.  The graphs belong to the
 * device's context: an application that resets a device (cudaDeviceReset)
 * calls lap5cg_release_graphs first.  One exception to "the caller owns every
 * buffer": cg_solve_classic_f64_noalloc uses a fixed 8.25 MiB __device__ array
 * of the library as scratch; the CUDA runtime commits it on a device when it
 * loads the library's module there (with lazy module loading, at the first
 * call into the library on that device, not at dlopen).
 *
 * Ordering: every call is asynchronous on the given CUDA stream (a
 * cudaStream_t passed as void*; NULL = the legacy default stream).  The return
 * value reports host-side argument validation and launch errors only; solve
 * outcomes are written to the device-side lap5cg_info once the stream reaches
 * them.  No entry point synchronises the device.
 *
 * Errors: negative return values are errors, 0 is success.  No C++ exception
 * crosses this interface.
 */
#ifndef LAP5CG_H
#define LAP5CG_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define LAP5CG_API __attribute__((visibility("default")))
#else
#define LAP5CG_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

/* Status codes, used both as return values and in lap5cg_info.status. */
typedef enum {
  LAP5CG_OK = 0,                 /* converged (or nothing to do) */
  LAP5CG_NOT_CONVERGED = 1,      /* maxit reached before the tolerance */
  LAP5CG_ERR_INVALID_ARG = -1,   /* rejected on the host before launch */
  LAP5CG_ERR_CUDA = -2,          /* a CUDA runtime call failed */
  LAP5CG_ERR_BREAKDOWN = -3,     /* (p,Ap) <= 0 (classic) or the NewCG alpha denominator <= 0 */
  LAP5CG_ERR_SYNC_TIMEOUT = -4,  /* a device-side grid barrier exceeded its time limit */
  LAP5CG_ERR_NONFINITE = -5,     /* a reduction produced Inf or NaN (e.g. NaN in b) */
  LAP5CG_ERR_UNSUPPORTED = -6,   /* valid but not supported combination */
  LAP5CG_ERR_WORKSPACE = -7      /* workspace missing, too small or misaligned */
} lap5cg_status;

/* Element types of lap5_apply. */
typedef enum { LAP5CG_DT_F64 = 0, LAP5CG_DT_F32 = 1, LAP5CG_DT_BF16 = 2 } lap5cg_dtype;

/* Algorithm 1 or Algorithm 2. */
typedef enum { LAP5CG_CLASSIC = 0, LAP5CG_NEWCG = 1 } lap5cg_variant;

/* Precision of a solve.
 *   F64      : b, x binary64; all arithmetic binary64.
 *   F32      : b, x binary32; arithmetic binary32, dot products accumulated
 *              with compensated (Dot2) summation, scalars in binary64.
 *   IR_F32   : b, x binary64.  Outer FP64 iterative refinement (residual
 *              b - A x, update x += d and their dot products in binary64)
 *              around an inner classic CG stored and computed in binary32.
 *   IR_BF16PR: as IR_F32 but the inner p and r are stored as bf16 (round to
 *              nearest even); inner arithmetic binary32.
 *   MG_F32:    preconditioned CG (Algorithm 1 with M; the cited pipelined CG
 *              takes a general M, the paper uses M = I) in binary64, M^-1 one
 *              geometric multigrid V(nu, nu) cycle in binary32: levels
 *              (nx, ny) -> ((nx-1)/2, (ny-1)/2), bilinear prolongation P,
 *              restriction P^T, the 5-point mask on every level, damped Jacobi
 *              (omega = 4/5) smoothing.  b and x binary64.  LAP5CG_CLASSIC:
 *              PCG; LAP5CG_NEWCG: LAP5CG_ERR_UNSUPPORTED (the pipelined
 *              recurrences need an exactly linear M; see MG_F64).
 *   MG_F64:    the same with the V-cycle in binary64; LAP5CG_NEWCG runs the
 *              pipelined form (Algorithm 2 with M: one fused pass and one grid
 *              reduction per iteration besides M^-1).
 *              MG_F32 / MG_F64 with LAP5CG_CLASSIC run as a CUDA graph (one
 *              kernel per pass, the iterations looped on the device by a
 *              conditional node; cached, see Ownership), or as one persistent
 *              kernel when the stream is being captured into the caller's
 *              graph; the pipelined form is always one persistent kernel.
 *              Concurrent calls must not share a workspace. */
typedef enum {
  LAP5CG_PREC_F64 = 0, LAP5CG_PREC_F32 = 1, LAP5CG_PREC_IR_F32 = 2, LAP5CG_PREC_IR_BF16PR = 3,
  LAP5CG_PREC_MG_F32 = 4, LAP5CG_PREC_MG_F64 = 5
} lap5cg_precision;

/* Per-solve outcome, written on the device (one entry per right-hand side or
 * per batched instance). */
typedef struct {
  int32_t status;           /* lap5cg_status */
  int32_t iters;            /* x updates done (IR: total inner iterations) */
  int32_t outer_iters;      /* IR refinement steps; 0 for F64/F32 */
  int32_t pad;
  double relres_recursive;  /* sqrt((r,r)/(b,b)) of the recurrence residual at exit */
  double relres_true;       /* ||b - A x|| / ||b|| recomputed at exit (NaN if disabled) */
} lap5cg_info;

/* Optional tuning and behaviour knobs.  Pass NULL for defaults, or fill a
 * struct with lap5cg_opts_default() and change fields. */
typedef struct {
  int32_t rr_period;        /* NewCG residual replacement every rr_period updates; 0 = off */
  int32_t store_z;          /* classic: 1 stores z = A p (fewer FP64 ops), 0 recomputes A p
                               in the update pass (fewer bytes), -1 = choose by precision */
  int32_t ctas;             /* persistent CTAs; 0 = choose from size and occupancy */
  int32_t warps_per_cta;    /* 1..16; 0 = default (4; batched and cluster-resident solves: 8;
                               multigrid solves: 16) */
  int32_t min_rows;         /* minimum rows per warp unit; 0 = default (2) */
  int32_t true_residual;    /* 1 (default) recompute ||b - A x|| at exit, 0 skip */
  int32_t maxit_inner;      /* IR: inner iteration cap per refinement step; 0 = default
                               (IR_F32: 4 (nx + ny) + 50; IR_BF16PR: 2 (nx + ny) + 50) */
  int32_t max_outer;        /* IR: refinement step cap; 0 = default (60) */
  double tol_inner;         /* IR: inner relative tolerance; <= 0 = default (1e-4 F32, 1e-2 BF16) */
  double timeout_s;         /* device barrier time limit in seconds; <= 0 = default (2 s) */
  double* history;          /* optional device array of maxit+1 doubles: recursive
                               relative residual after each update; NULL = off
                               (single solves only) */
  int32_t team_ctas;        /* cg_solve_batched: CTAs per instance team (one thread-block
                               cluster: 1, 2, 4, 8 or 16); 0 = default (8).  For batched
                               solves `ctas` caps the total CTAs.  cg_solve of a grid that
                               fits in one cluster's shared memory (`resident`): the cluster
                               size (1, 2, 4, 8 or 16; other values: 16), at most one CTA a
                               row. */
  int32_t ring_slots;       /* rows each warp keeps in flight in its shared-memory ring
                               (bulk asynchronous copies): 0 = automatic (on when the warp
                               units are at least 8 rows tall),
                               3..8 = that many, < 0 = no ring (rows loaded into registers) */
  int32_t resident;         /* F64 / F32 solves of grids that fit in the shared memory of one
                               thread-block cluster (about 250 x 250 binary64): 0 = solve them
                               there (default, when ring_slots == 0 and rr_period == 0),
                               < 0 = always use the streaming kernels */
  int32_t lane_vec;         /* columns each lane owns in its warp's strip.
                               Binary32 passes (F32 classic; the inner passes of IR_F32 /
                               IR_BF16PR): 4 or 8; 0 = automatic (8 when nx >= 1024 and the
                               ring is used).  8 needs the classic variant and the
                               shared-memory ring (ring_slots > 0, or automatic with units at
                               least 8 rows tall), and store_z <= 0 for IR.
                               F64: 2 or 4; 0 = automatic (4 for classic CG with the ring when
                               ld is a multiple of 4, else 2).  4 needs the classic variant,
                               the ring and ld a multiple of 4; the reproducible mode takes 2.
                               Other combinations: LAP5CG_ERR_UNSUPPORTED.  Multigrid and
                               batched solves ignore it. */
  int32_t reproducible;     /* cg_solve, F64 (classic and NewCG): 1 = dot products whose value
                               does not depend on the launch configuration (CTAs, warps, ring,
                               unit sizes): each is the exact sum of fixed 2-column x 16-row
                               block values (row value fma(a1, b1, a0*b0), a pairwise tree over
                               the 16 rows), rounded once; vector updates are single-rounding
                               fused multiply-adds.  Equal inputs and options other than the
                               launch parameters give bit-identical results.  0 = the default
                               fixed-order partial sums.  Other precisions, grids of 2^36
                               points or more and batched solves: LAP5CG_ERR_UNSUPPORTED. */
  int32_t mg_nu;            /* MG_F32 / MG_F64: smoothing sweeps before and after the coarse
                               correction; 0 = default (2) */
  int32_t mg_levels;        /* MG_F32 / MG_F64: at most this many grids; 0 = as many as the
                               sides allow */
  int32_t mg_coarse_sweeps; /* MG_F32 / MG_F64: damped Jacobi sweeps on the coarsest grid;
                               0 = default (8) */
  int32_t stabilized;       /* cg_solve, NEWCG, F64 / F32: 1 = alpha = gamma / (p, A p) with
                               (p, A p) = delta + 2 beta (r, q_old) + beta^2 (p_old, q_old) formed
                               from dot products of the current vectors, reduced together with
                               gamma and delta (still one reduction per iteration), instead of
                               Algorithm 2's recurrence alpha = 1/(delta/gamma - beta/alpha_old).
                               Equal in exact arithmetic; the recurrence assumes orthogonal
                               consecutive residuals and breaks down near the attainable accuracy
                               (e.g. above 1e-10 at 8192 x 8192).  Two more multiply-adds a point.
                               0 = Algorithm 2 (default).  CLASSIC: LAP5CG_ERR_INVALID_ARG; other
                               precisions, reproducible mode and batched solves:
                               LAP5CG_ERR_UNSUPPORTED.  Solves always take the streaming kernels. */
} lap5cg_opts;

/* Fill *o with the defaults above. */
LAP5CG_API void lap5cg_opts_default(lap5cg_opts* o);

/* Human-readable text of a status code (static storage). */
LAP5CG_API const char* lap5cg_status_string(int status);

/*
 * y = A x, the Sec. II-B mask with zero Dirichlet boundary, in the fixed add
 * order y = 4*xC - xW - xE - xS - xN (W/E: i-1/i+1, S/N: j-1/j+1).
 *   dtype F64: binary64; F32: binary32; BF16: bf16 in and out, binary32
 *   arithmetic, result rounded to nearest even.
 *   x, y: device pointers to ny*ld elements each; must not overlap.
 * Returns LAP5CG_OK, LAP5CG_ERR_INVALID_ARG (nx or ny < 1, ld < nx, NULL
 * pointers, unknown dtype) or LAP5CG_ERR_CUDA.
 */
LAP5CG_API int lap5_apply(int nx, int ny, int ld, int dtype, const void* x, void* y, void* stream);

/*
 * Bytes of device workspace cg_solve needs for this shape, variant and
 * precision (for nrhs right-hand sides solved one after another the workspace
 * is reused, so nrhs does not change the size).  Returns 0 for invalid
 * arguments.
 */
LAP5CG_API size_t cg_workspace_size(int nx, int ny, int ld, int variant, int precision, int nrhs);

/*
 * Solve A x = b (Algorithm 1 or 2) in one persistent kernel per right-hand side.
 *   b, x     : device pointers, nrhs grids of ny*ld elements each, stored one
 *              after another (right-hand side k at offset k*ny*ld).  Element
 *              type: binary64 for F64/IR_*, binary32 for F32.  On entry x is the
 *              initial guess x0 (zeros for the paper's setting); on exit the
 *              solution.  b and x must not overlap.
 *   tol      : stop when (r,r) <= tol^2 (b,b) (recursive residual); tol <= 0
 *              runs maxit updates.  IR: tol applies to the FP64 true residual.
 *   maxit    : maximum x updates (IR: maximum total inner iterations); >= 0.
 *   workspace: device buffer of at least cg_workspace_size() bytes, 256-byte
 *              aligned; contents on entry are irrelevant.
 *   info     : device pointer to nrhs lap5cg_info entries.
 *   opts     : NULL or tuning knobs (host pointer, read during the call).
 * b = 0 yields x = 0, iters = 0, LAP5CG_OK.  The convergence test and all
 * scalars stay on the device; no host synchronisation happens per iteration.
 * Returns LAP5CG_OK when every launch was enqueued, else an error code.
 */
LAP5CG_API int cg_solve(int nx, int ny, int ld, const void* b, void* x, double tol, int maxit,
             int variant, int precision, int nrhs, void* workspace, size_t ws_bytes,
             lap5cg_info* info, const lap5cg_opts* opts, void* stream);

/* Largest instance count one cg_solve_batched call accepts. */
#define LAP5CG_MAX_BATCH 1024

/*
 * Bytes of device workspace cg_solve_batched needs for these shapes (host
 * arrays of count entries).  Returns 0 for invalid arguments.
 */
LAP5CG_API size_t cg_batched_workspace_size(int count, const int* nx, const int* ny, const int* ld,
                                 int variant, int precision);

/*
 * Solve count independent systems A_k x_k = b_k of different shapes in one
 * persistent launch.  Each instance is solved by a team of CTAs forming one
 * thread-block cluster (cluster barrier, reductions through distributed shared
 * memory); teams take instances from a device-side queue ordered by estimated
 * work, largest first, so an instance that has converged stops and its team
 * takes the next one (per-instance convergence masking).  Per instance the
 * arithmetic is that of cg_solve (Algorithm 1 / 2, same precisions).
 *   count     : 1 .. LAP5CG_MAX_BATCH.
 *   nx, ny, ld: host arrays of count shapes; every ld must be a multiple of
 *               the lane vector width (2 for F64, 4 otherwise) and every b, x
 *               16-byte aligned (no staging in batched mode).
 *   b, x      : host arrays of count device pointers (element type as in
 *               cg_solve for the precision); x holds x0 on entry.
 *   info      : device pointer to count lap5cg_info entries (caller order).
 *   workspace : at least cg_batched_workspace_size() bytes, 256-byte aligned.
 * The host arrays are read during the call only; the call enqueues a few
 * table-fill kernels, a memset and the solver launch on the stream.
 * Returns LAP5CG_ERR_UNSUPPORTED for NEWCG with the IR precisions.
 */
LAP5CG_API int cg_solve_batched(int count, const int* nx, const int* ny, const int* ld,
                     const void* const* b, void* const* x, double tol, int maxit,
                     int variant, int precision, void* workspace, size_t ws_bytes,
                     lap5cg_info* info, const lap5cg_opts* opts, void* stream);

/*
 * Autotuner (launch parameters only; the arithmetic does not change).  Times
 * fixed-iteration solves (tol = 0, `iters` updates, x reset to 0 before each
 * trial) with CUDA events on `stream` and searches, by coordinate descent
 * starting from *opts, over warps_per_cta, ring_slots, min_rows and (classic
 * F64/F32) store_z.  On return *opts holds the fastest combination found and
 * *best_ms (if not NULL) its time.  Arguments as cg_solve; x is overwritten
 * (used as scratch); the call synchronises the stream.  No paper counterpart.
 */
LAP5CG_API int lap5cg_tune(int nx, int ny, int ld, const void* b, void* x, int variant, int precision, int iters,
                           void* workspace, size_t ws_bytes, lap5cg_info* info, lap5cg_opts* opts,
                           double* best_ms, void* stream);

/* The same for cg_solve_batched, over team_ctas, warps_per_cta, ring_slots and
 * min_rows; every x[k] is overwritten.  iters = 0: each trial solves every
 * instance to a relative residual of 1e-4 instead of a fixed iteration count,
 * so that larger instances weigh more, as in a real solve. */
LAP5CG_API int lap5cg_tune_batched(int count, const int* nx, const int* ny, const int* ld, const void* const* b,
                                   void* const* x, int variant, int precision, int iters, void* workspace,
                                   size_t ws_bytes, lap5cg_info* info, lap5cg_opts* opts, double* best_ms,
                                   void* stream);

/*
 * Measurement helper (no paper counterpart): the binary64 instruction rates of
 * the current GPU, in lane operations per second -- fused multiply-adds
 * (*fma_per_s) and additions (*add_per_s) -- from a throughput kernel with
 * eight independent dependency chains a thread and 64 warps on every SM,
 * timed with CUDA events on `stream` (best of five launches of about 40 ms
 * each; the GPU's clocks should be up, e.g. after other work).  The
 * binary64 solves are bound by this pipe rather than by memory bandwidth.
 * Synchronises the stream; allocates no device memory.
 * Returns LAP5CG_OK, LAP5CG_ERR_INVALID_ARG (NULL outputs) or LAP5CG_ERR_CUDA.
 */
LAP5CG_API int lap5cg_fp64_rate(double* fma_per_s, double* add_per_s, void* stream);

/*
 * Frees every cached graph of the classic multigrid-preconditioned solve, on
 * every device (see Ownership above).  Call it before resetting a device or
 * destroying its primary context: the cached graphs belong to that context.
 * A graph still running is freed by the driver when it completes.  The next
 * classic MG_F32 / MG_F64 solve of a shape builds its graph again.  Safe to
 * call from any host thread at any time (the cache has a lock); allocates
 * nothing.  Returns LAP5CG_OK, or LAP5CG_ERR_CUDA if a graph could not be
 * destroyed (the cache is emptied all the same).
 */
LAP5CG_API int lap5cg_release_graphs(void);

/* Largest ny*ld that cg_solve_classic_f64_noalloc accepts. */
#define LAP5CG_NOALLOC_MAX_POINTS 262144

/*
 * The binary64 classic CG solve (Algorithm 1, the arithmetic of cg_solve with
 * variant CLASSIC, precision F64, nrhs 1, default options, always on the
 * streaming kernels: grids that cg_solve would solve in one cluster's shared
 * memory take the streaming path here, so iteration counts and low-order bits
 * may differ from cg_solve on such grids) for callers that cannot allocate
 * device memory: its scratch space is a fixed array inside this library, so
 * no workspace argument is needed.  The paper has no counterpart; this entry
 * point exists for the library's users.
 *
 * Who needs it: applications that fix their device-memory budget at start-up
 * and forbid allocation afterwards (real-time and safety-certified code),
 * plug-ins running inside a host framework that owns every device allocation
 * through its own pool, and latency-critical loops that cannot afford the
 * device synchronisation a cudaMalloc/cudaFree may imply.
 *
 * Limits and behaviour:
 *   - ny*ld <= LAP5CG_NOALLOC_MAX_POINTS (e.g. 512 x 512); larger grids are
 *     rejected with LAP5CG_ERR_INVALID_ARG.  ld must be even and b, x 16-byte
 *     aligned (LAP5CG_ERR_INVALID_ARG otherwise): there is no staging space.
 *   - The scratch array (8.25 MiB) is a static __device__ object: every GPU
 *     that loads this library holds it until the process exits.
 *   - Every call looks up the array's device address on the current device
 *     (cudaGetSymbolAddress; nothing is cached, so the address stays right
 *     after a device reset reloads the module).  The first call on a device
 *     may load the module and commit the array: make one warm-up call per
 *     device at start-up, before any stream capture, so that a fixed memory
 *     budget sees the array from the start.
 *   - The device is the current one: b, x and info must live on it.
 *   - All calls share the one array and the solver re-initialises what must
 *     start at zero, but calls that overlap on the GPU (different streams, or
 *     different host threads, on the same device) race on it: serialise them.
 *   - Calls no cudaMalloc, cudaFree or other allocating routine.
 * b, x, tol, maxit, info (one entry) and stream are as in cg_solve.
 */
LAP5CG_API int cg_solve_classic_f64_noalloc(int nx, int ny, int ld, const double* b, double* x, double tol,
                                            int maxit, lap5cg_info* info, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* LAP5CG_H */
