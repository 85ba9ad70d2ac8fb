/*
 * lap5_oracle.c -- plain, slow, obviously correct CPU oracle for matrix-free
 * conjugate gradient on the 2D Dirichlet 5-point Laplacian
 * (arxiv 1803.03797, "Efficient FPGA Implementation of Conjugate Gradient
 * Methods for Laplacian System using HLS").
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path (the CUDA library and
 * its Python binding) may call, link or include this file.  It shares no code,
 * header, table or helper with the GPU path.  Only the test suite, the smoke
 * check and the CPU-baseline leg of the benchmark use it.
 *
 * Build: gcc -O2 -std=c11 -ffp-contract=off -fPIC -shared (see oracle/build.py).
 * -ffp-contract=off matters: every a*b+c below is two roundings, as written.
 *
 * Conventions (shared with the public C-ABI only by meaning, not by code):
 *   grid: nx columns (i, fastest) by ny rows (j); element (i,j) at j*ld + i,
 *   ld >= nx; the Dirichlet boundary is implicit zeros, never stored.
 *   A = the paper's 3x3 mask [0 -1 0; -1 4 -1; 0 -1 0] (Sec. II-B), no 1/h^2.
 *
 * Readings of the paper taken here:
 *   - stencil add order: acc = 4*xC; acc -= xW; acc -= xE; acc -= xS; acc -= xN
 *     (W = i-1, E = i+1, S = j-1, N = j+1).  The paper fixes only the mask.
 *   - Alg. 2 garbles: "r = r + alpha*s" read as r = r - alpha*q;
 *     "w = w + alpha*z" read as w = w - alpha*z; the unbalanced alpha update
 *     read as alpha = 1/(delta/gamma - beta/alpha_old); the delta of the
 *     first alpha is delta_new.
 *     These follow the cited Ghysels-Vanroose pipelined CG with M = I.
 *   - stopping test: recursive gamma = (r,r) <= tol^2 (b,b); tol <= 0 means
 *     "never stop early" (threshold 0).  iters = number of x updates.
 *   - b = 0 gives x = 0, iters = 0, status OK.
 *   - breakdown: (p,Ap) <= 0 (classic) or delta/gamma - beta/alpha_old <= 0
 *     (NewCG), or any non-finite reduction.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* Timing build (oracle/build.py, -fopenmp -DORA_OMP): the row loops of the
 * binary64 stencil and vector helpers run on all threads, and ora_dot_f64 sums
 * per-thread partials of contiguous row blocks in thread order.  Only the
 * benchmark's CPU-baseline timing loads that build; the parity build (no
 * ORA_OMP) is the plain sequential code below, and ORA_ROWS is empty there. */
#ifdef ORA_OMP
#include <omp.h>
#define ORA_ROWS _Pragma("omp parallel for schedule(static)")
#else
#define ORA_ROWS
#endif

enum { ORA_OK = 0, ORA_NOT_CONVERGED = 1, ORA_ERR_INVALID_ARG = -1,
       ORA_ERR_BREAKDOWN = -3, ORA_ERR_NONFINITE = -5 };

typedef struct {
  int32_t status;
  int32_t iters;        /* x updates (classic/NewCG), total inner iterations (IR) */
  int32_t outer_iters;  /* refinement steps (IR), 0 otherwise */
  int32_t pad;
  double relres_recursive;  /* sqrt(gamma_last / (b,b)) */
  double relres_true;       /* ||b - A x|| / ||b|| recomputed at the end */
} ora_info;

/* Optional per-iteration record, used by the invariant tests.  Every pointer
 * may be NULL.  Vector traces hold ntrace snapshots of ny*ld doubles each:
 * snapshot k is taken after k x-updates (k = 0 is the initial state).  For
 * classic CG, p[k] is the direction used by update k+1; for NewCG, p[k], q[k],
 * z[k] are the values used by update k+1 and w[k] the w after update k. */
typedef struct {
  double* x; double* r; double* p; double* w; double* q; double* z;
  double* alpha;   /* [ntrace] alpha of update k+1 */
  double* beta;    /* [ntrace] beta used to form p of update k+1 */
  double* relres;  /* [maxit+1] sqrt(gamma_k/(b,b)) after k updates */
  int32_t ntrace;
  int32_t pad;
} ora_trace;

/* ------------------------------------------------------------------ */
/* Stencil y = A x (Sec. II-B mask; fixed add order).                   */
/* ------------------------------------------------------------------ */

static double at64(const double* x, int nx, int ny, int ld, int i, int j) {
  if (i < 0 || i >= nx || j < 0 || j >= ny) return 0.0;   /* zero Dirichlet */
  return x[(size_t)j * ld + i];
}

void ora_lap5_apply_f64(int nx, int ny, int ld, const double* x, double* y) {
  ORA_ROWS
  for (int j = 0; j < ny; ++j)
    for (int i = 0; i < nx; ++i) {
      double acc = 4.0 * at64(x, nx, ny, ld, i, j);
      acc -= at64(x, nx, ny, ld, i - 1, j);
      acc -= at64(x, nx, ny, ld, i + 1, j);
      acc -= at64(x, nx, ny, ld, i, j - 1);
      acc -= at64(x, nx, ny, ld, i, j + 1);
      y[(size_t)j * ld + i] = acc;
    }
}

static float at32(const float* x, int nx, int ny, int ld, int i, int j) {
  if (i < 0 || i >= nx || j < 0 || j >= ny) return 0.0f;
  return x[(size_t)j * ld + i];
}

/* Same stencil with every operation rounded to binary32. */
void ora_lap5_apply_f32(int nx, int ny, int ld, const float* x, float* y) {
  for (int j = 0; j < ny; ++j)
    for (int i = 0; i < nx; ++i) {
      float acc = 4.0f * at32(x, nx, ny, ld, i, j);
      acc -= at32(x, nx, ny, ld, i - 1, j);
      acc -= at32(x, nx, ny, ld, i + 1, j);
      acc -= at32(x, nx, ny, ld, i, j - 1);
      acc -= at32(x, nx, ny, ld, i, j + 1);
      y[(size_t)j * ld + i] = acc;
    }
}

/* bfloat16 <-> binary32.  bf16 is the upper half of a binary32 word, so the
 * widening is exact; narrowing rounds to nearest, ties to even. */
static float bf16_to_f32(uint16_t h) {
  uint32_t u = (uint32_t)h << 16; float f; memcpy(&f, &u, 4); return f;
}
static uint16_t f32_to_bf16(float f) {
  uint32_t u; memcpy(&u, &f, 4);
  if ((u & 0x7fffffffu) > 0x7f800000u) return (uint16_t)((u >> 16) | 0x0040u); /* NaN stays NaN */
  uint32_t keep = u >> 16;
  uint32_t rest = u & 0xffffu;
  /* round half to even on the discarded 16 bits */
  if (rest > 0x8000u || (rest == 0x8000u && (keep & 1u))) keep += 1u;
  return (uint16_t)keep;
}

uint16_t ora_f32_to_bf16(float f) { return f32_to_bf16(f); }
float ora_bf16_to_f32(uint16_t h) { return bf16_to_f32(h); }

/* bf16 storage, binary32 arithmetic in the fixed order, result rounded to bf16. */
void ora_lap5_apply_bf16(int nx, int ny, int ld, const uint16_t* x, uint16_t* y) {
  for (int j = 0; j < ny; ++j)
    for (int i = 0; i < nx; ++i) {
#define XB(ii, jj) (((ii) < 0 || (ii) >= nx || (jj) < 0 || (jj) >= ny) ? 0.0f : bf16_to_f32(x[(size_t)(jj) * ld + (ii)]))
      float acc = 4.0f * XB(i, j);
      acc -= XB(i - 1, j);
      acc -= XB(i + 1, j);
      acc -= XB(i, j - 1);
      acc -= XB(i, j + 1);
#undef XB
      y[(size_t)j * ld + i] = f32_to_bf16(acc);
    }
}

/* ------------------------------------------------------------------ */
/* Vector helpers over the nx-by-ny interior (padding columns ignored). */
/* ------------------------------------------------------------------ */

/* (a, b) summed in index order (row by row, i fastest), binary64. */
double ora_dot_f64(int nx, int ny, int ld, const double* a, const double* b) {
#ifdef ORA_OMP
  double part[256];
  int used = 1;
#pragma omp parallel num_threads(omp_get_max_threads() < 256 ? omp_get_max_threads() : 256)
  {
    const int t = omp_get_thread_num(), T = omp_get_num_threads();
    const int j0 = (int)((long long)ny * t / T), j1 = (int)((long long)ny * (t + 1) / T);
    double s = 0.0;
    for (int j = j0; j < j1; ++j)
      for (int i = 0; i < nx; ++i) s += a[(size_t)j * ld + i] * b[(size_t)j * ld + i];
    part[t] = s;
    if (t == 0) used = T;
  }
  double s = 0.0;
  for (int t = 0; t < used; ++t) s += part[t];
  return s;
#else
  double s = 0.0;
  for (int j = 0; j < ny; ++j)
    for (int i = 0; i < nx; ++i) s += a[(size_t)j * ld + i] * b[(size_t)j * ld + i];
  return s;
#endif
}

/* threads of the timing build (1 in the parity build) */
int ora_threads(void) {
#ifdef ORA_OMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

static void axpy64(int nx, int ny, int ld, double* y, double a, const double* x) {
  ORA_ROWS
  for (int j = 0; j < ny; ++j)
    for (int i = 0; i < nx; ++i) y[(size_t)j * ld + i] = y[(size_t)j * ld + i] + a * x[(size_t)j * ld + i];
}

/* y = x + beta * y */
static void xpby64(int nx, int ny, int ld, const double* x, double beta, double* y) {
  ORA_ROWS
  for (int j = 0; j < ny; ++j)
    for (int i = 0; i < nx; ++i) y[(size_t)j * ld + i] = x[(size_t)j * ld + i] + beta * y[(size_t)j * ld + i];
}

static void copy64(int nx, int ny, int ld, double* y, const double* x) {
  ORA_ROWS
  for (int j = 0; j < ny; ++j) memcpy(y + (size_t)j * ld, x + (size_t)j * ld, sizeof(double) * (size_t)nx);
}

static void zero64(int nx, int ny, int ld, double* y) {
  ORA_ROWS
  for (int j = 0; j < ny; ++j) memset(y + (size_t)j * ld, 0, sizeof(double) * (size_t)nx);
}

/* r = b - A x */
static void residual64(int nx, int ny, int ld, const double* b, const double* x, double* r) {
  ora_lap5_apply_f64(nx, ny, ld, x, r);
  ORA_ROWS
  for (int j = 0; j < ny; ++j)
    for (int i = 0; i < nx; ++i) r[(size_t)j * ld + i] = b[(size_t)j * ld + i] - r[(size_t)j * ld + i];
}

static double true_relres(int nx, int ny, int ld, const double* b, const double* x, double bb) {
  size_t n = (size_t)ny * ld;
  double* r = (double*)calloc(n, sizeof(double));
  if (!r) return NAN;
  residual64(nx, ny, ld, b, x, r);
  double rr = ora_dot_f64(nx, ny, ld, r, r);
  free(r);
  return sqrt(rr / bb);
}

static void snap(double* dst, int k, int ntrace, size_t n, const double* src) {
  if (dst && k >= 0 && k < ntrace) memcpy(dst + (size_t)k * n, src, n * sizeof(double));
}

static int arg_ok(int nx, int ny, int ld, int maxit) {
  return nx >= 1 && ny >= 1 && ld >= nx && maxit >= 0;
}

/* ------------------------------------------------------------------ */
/* Algorithm 1 (classic CG), with an initial guess x0 allowed.           */
/* ------------------------------------------------------------------ */
int ora_cg_classic(int nx, int ny, int ld, const double* b, double* x, double tol, int maxit,
                   ora_trace* tr, ora_info* info) {
  ora_info inf; memset(&inf, 0, sizeof inf);
  if (!arg_ok(nx, ny, ld, maxit) || !b || !x) { inf.status = ORA_ERR_INVALID_ARG; if (info) *info = inf; return inf.status; }
  const size_t n = (size_t)ny * ld;
  const int nt = tr ? tr->ntrace : 0;
  double bb = ora_dot_f64(nx, ny, ld, b, b);
  if (!isfinite(bb)) { inf.status = ORA_ERR_NONFINITE; inf.relres_recursive = NAN; inf.relres_true = NAN; if (info) *info = inf; return inf.status; }
  if (bb == 0.0) {  /* A x = 0 has the unique solution x = 0 */
    zero64(nx, ny, ld, x);
    inf.status = ORA_OK; if (info) *info = inf; return inf.status;
  }
  const double thr = tol > 0.0 ? tol * tol * bb : 0.0;
  double* r = (double*)calloc(n, sizeof(double));
  double* p = (double*)calloc(n, sizeof(double));
  double* z = (double*)calloc(n, sizeof(double));
  if (!r || !p || !z) { free(r); free(p); free(z); inf.status = ORA_ERR_INVALID_ARG; if (info) *info = inf; return inf.status; }

  residual64(nx, ny, ld, b, x, r);                 /* r_old = b - A x0 (= b for x0 = 0) */
  double gamma = ora_dot_f64(nx, ny, ld, r, r);    /* (r_old, r_old) */
  copy64(nx, ny, ld, p, r);                        /* p = r_old */
  if (tr && tr->relres) tr->relres[0] = sqrt(gamma / bb);
  if (tr) { snap(tr->x, 0, nt, n, x); snap(tr->r, 0, nt, n, r); snap(tr->p, 0, nt, n, p);
            if (tr->beta && nt > 0) tr->beta[0] = 0.0; }
  int status = ORA_NOT_CONVERGED, k = 0;
  if (!isfinite(gamma)) status = ORA_ERR_NONFINITE;
  else if (gamma <= thr) status = ORA_OK;
  while (status == ORA_NOT_CONVERGED && k < maxit) {
    ora_lap5_apply_f64(nx, ny, ld, p, z);            /* z = A p */
    double pz = ora_dot_f64(nx, ny, ld, z, p);       /* (z, p) */
    if (!(pz > 0.0) || !isfinite(pz)) { status = ORA_ERR_BREAKDOWN; break; }
    double alpha = gamma / pz;
    if (tr && tr->alpha && k < nt) tr->alpha[k] = alpha;
    axpy64(nx, ny, ld, x, alpha, p);                 /* x = x + alpha p */
    axpy64(nx, ny, ld, r, -alpha, z);                /* r = r_old - alpha z */
    double gnew = ora_dot_f64(nx, ny, ld, r, r);     /* (r, r) */
    ++k;
    if (tr) { snap(tr->x, k, nt, n, x); snap(tr->r, k, nt, n, r); if (tr->relres) tr->relres[k] = sqrt(gnew / bb); }
    if (!isfinite(gnew)) { status = ORA_ERR_NONFINITE; gamma = gnew; break; }
    double beta = gnew / gamma;                      /* (r,r)/(r_old,r_old) */
    gamma = gnew;                                    /* r_old = r */
    if (gnew <= thr) { status = ORA_OK; break; }
    xpby64(nx, ny, ld, r, beta, p);                  /* p = r + beta p */
    if (tr) { snap(tr->p, k, nt, n, p); if (tr->beta && k < nt) tr->beta[k] = beta; }
  }
  inf.status = status; inf.iters = k;
  inf.relres_recursive = sqrt(gamma / bb);
  inf.relres_true = true_relres(nx, ny, ld, b, x, bb);
  free(r); free(p); free(z);
  if (info) *info = inf;
  return status;
}

/* ------------------------------------------------------------------ */
/* Algorithm 2 (NewCG = pipelined CG of Ghysels & Vanroose, M = I).      */
/* rr_period > 0 enables residual replacement every rr_period updates:   */
/* r = b - A x, w = A r, q = A p, z = A q are recomputed from x and p.   */
/* ------------------------------------------------------------------ */
/* stable = 1 forms alpha from (p, A p) of the new direction p = r + beta p_old
 * expanded into dot products of the current vectors,
 *   (p, A p) = delta + 2 beta (r, q_old) + beta^2 (p_old, q_old),
 * instead of the scalar recurrence alpha = 1/(delta/gamma - beta/alpha_old).
 * The two are equal in exact arithmetic ((r, q_old) = -gamma/alpha_old and
 * (p_old, q_old) = gamma_old/alpha_old there); the recurrence assumes that
 * consecutive residuals are orthogonal, which rounding undoes once the
 * residual nears its attainable accuracy -- alpha then drifts by percents and
 * the iteration breaks down.  The extra dots need no extra synchronisation
 * (the predict-and-recompute idea of Chen & Carson, SIAM J. Sci. Comput. 2020:
 * form the needed inner products from the vectors at hand). */
static int cg_newcg_impl(int nx, int ny, int ld, const double* b, double* x, double tol, int maxit,
                         int rr_period, int stable, ora_trace* tr, ora_info* info);

int ora_cg_newcg(int nx, int ny, int ld, const double* b, double* x, double tol, int maxit,
                 int rr_period, ora_trace* tr, ora_info* info) {
  return cg_newcg_impl(nx, ny, ld, b, x, tol, maxit, rr_period, 0, tr, info);
}

int ora_cg_newcg_stable(int nx, int ny, int ld, const double* b, double* x, double tol, int maxit,
                        int rr_period, ora_trace* tr, ora_info* info) {
  return cg_newcg_impl(nx, ny, ld, b, x, tol, maxit, rr_period, 1, tr, info);
}

static int cg_newcg_impl(int nx, int ny, int ld, const double* b, double* x, double tol, int maxit,
                         int rr_period, int stable, ora_trace* tr, ora_info* info) {
  ora_info inf; memset(&inf, 0, sizeof inf);
  if (!arg_ok(nx, ny, ld, maxit) || !b || !x || rr_period < 0) { inf.status = ORA_ERR_INVALID_ARG; if (info) *info = inf; return inf.status; }
  const size_t n = (size_t)ny * ld;
  const int nt = tr ? tr->ntrace : 0;
  double bb = ora_dot_f64(nx, ny, ld, b, b);
  if (!isfinite(bb)) { inf.status = ORA_ERR_NONFINITE; inf.relres_recursive = NAN; inf.relres_true = NAN; if (info) *info = inf; return inf.status; }
  if (bb == 0.0) { zero64(nx, ny, ld, x); inf.status = ORA_OK; if (info) *info = inf; return inf.status; }
  const double thr = tol > 0.0 ? tol * tol * bb : 0.0;
  double *r = calloc(n, 8), *w = calloc(n, 8), *nv = calloc(n, 8), *z = calloc(n, 8), *q = calloc(n, 8), *p = calloc(n, 8);
  if (!r || !w || !nv || !z || !q || !p) { free(r); free(w); free(nv); free(z); free(q); free(p); inf.status = ORA_ERR_INVALID_ARG; if (info) *info = inf; return inf.status; }

  int status = ORA_NOT_CONVERGED, k = 0;
  residual64(nx, ny, ld, b, x, r);                    /* r = b - A x */
  ora_lap5_apply_f64(nx, ny, ld, r, w);               /* w = A r */
  double gamma = ora_dot_f64(nx, ny, ld, r, r);       /* gamma = (r, r) */
  if (tr && tr->relres) tr->relres[0] = sqrt(gamma / bb);
  if (tr) { snap(tr->x, 0, nt, n, x); snap(tr->r, 0, nt, n, r); snap(tr->w, 0, nt, n, w); }
  double alpha = 0.0;
  if (!isfinite(gamma)) status = ORA_ERR_NONFINITE;
  else if (gamma <= thr) status = ORA_OK;
  else if (maxit > 0) {
    double delta = ora_dot_f64(nx, ny, ld, w, r);     /* delta = (w, r) */
    ora_lap5_apply_f64(nx, ny, ld, w, nv);            /* n = A w */
    if (!(delta > 0.0) || !isfinite(delta)) status = ORA_ERR_BREAKDOWN;
    else {
      alpha = gamma / delta;                          /* alpha = gamma / delta (beta = 0) */
      copy64(nx, ny, ld, z, nv);                      /* z = n, q = w, p = r */
      copy64(nx, ny, ld, q, w);
      copy64(nx, ny, ld, p, r);
      if (tr) { snap(tr->p, 0, nt, n, p); snap(tr->q, 0, nt, n, q); snap(tr->z, 0, nt, n, z);
                if (tr->alpha && nt > 0) tr->alpha[0] = alpha;
                if (tr->beta && nt > 0) tr->beta[0] = 0.0; }
      axpy64(nx, ny, ld, x, alpha, p);                /* x = x + alpha p */
      axpy64(nx, ny, ld, r, -alpha, q);               /* r = r - alpha q (printed r + alpha s) */
      axpy64(nx, ny, ld, w, -alpha, z);               /* w = w - alpha z (printed w + alpha z) */
      k = 1;
      if (tr) { snap(tr->x, 1, nt, n, x); snap(tr->r, 1, nt, n, r); snap(tr->w, 1, nt, n, w); }
    }
  }
  while (status == ORA_NOT_CONVERGED && k >= 1) {
    if (rr_period > 0 && k % rr_period == 0) {        /* residual replacement */
      residual64(nx, ny, ld, b, x, r);
      ora_lap5_apply_f64(nx, ny, ld, r, w);
      ora_lap5_apply_f64(nx, ny, ld, p, q);
      ora_lap5_apply_f64(nx, ny, ld, q, z);
    }
    double gamma_old = gamma;                         /* gamma_old = gamma */
    gamma = ora_dot_f64(nx, ny, ld, r, r);            /* gamma = (r, r) */
    if (tr && tr->relres) tr->relres[k] = sqrt(gamma / bb);
    if (!isfinite(gamma)) { status = ORA_ERR_NONFINITE; break; }
    if (gamma <= thr) { status = ORA_OK; break; }
    if (k >= maxit) break;
    double delta = ora_dot_f64(nx, ny, ld, w, r);     /* delta = (w, r) */
    ora_lap5_apply_f64(nx, ny, ld, w, nv);            /* n = A w */
    double beta = gamma / gamma_old;                  /* beta = gamma / gamma_old */
    if (stable) {                                     /* (p, A p) from the current vectors */
      double eps = ora_dot_f64(nx, ny, ld, r, q);     /* (r, q_old) */
      double mu = ora_dot_f64(nx, ny, ld, p, q);      /* (p_old, q_old) */
      double pap = (delta + (2.0 * beta) * eps) + (beta * beta) * mu;
      if (!(pap > 0.0) || !isfinite(pap)) { status = ORA_ERR_BREAKDOWN; break; }
      alpha = gamma / pap;
    } else {
      double denom = delta / gamma - beta / alpha;    /* de-garbled alpha update */
      if (!(denom > 0.0) || !isfinite(denom)) { status = ORA_ERR_BREAKDOWN; break; }
      alpha = 1.0 / denom;
    }
    xpby64(nx, ny, ld, nv, beta, z);                  /* z = n + beta z */
    xpby64(nx, ny, ld, w, beta, q);                   /* q = w + beta q */
    xpby64(nx, ny, ld, r, beta, p);                   /* p = r + beta p */
    if (tr) { snap(tr->p, k, nt, n, p); snap(tr->q, k, nt, n, q); snap(tr->z, k, nt, n, z);
              if (tr->alpha && k < nt) tr->alpha[k] = alpha;
              if (tr->beta && k < nt) tr->beta[k] = beta; }
    axpy64(nx, ny, ld, x, alpha, p);                  /* x = x + alpha p */
    axpy64(nx, ny, ld, r, -alpha, q);                 /* r = r - alpha q */
    axpy64(nx, ny, ld, w, -alpha, z);                 /* w = w - alpha z */
    ++k;
    if (tr) { snap(tr->x, k, nt, n, x); snap(tr->r, k, nt, n, r); snap(tr->w, k, nt, n, w); }
  }
  inf.status = status; inf.iters = k;
  inf.relres_recursive = sqrt(gamma / bb);
  inf.relres_true = true_relres(nx, ny, ld, b, x, bb);
  free(r); free(w); free(nv); free(z); free(q); free(p);
  if (info) *info = inf;
  return status;
}

/* ------------------------------------------------------------------ */
/* Reproducible dot product: the building blocks.  The paper accumulates  */
/* in fixed point because floating-point addition is not associative and  */
/* so would tie the result to one order of operations (Sec. III, Sec.     */
/* II-C-1: the multiplier-adder tree).  Reading taken here: the value of  */
/* (a, b) is defined independently of how the grid is split:              */
/*  1. blocks of 2 columns x 16 rows aligned at column 2c and row 16t;     */
/*     points outside the grid have a = b = 0;                            */
/*  2. the row value of a block is fma(a1, b1, a0*b0) (columns 2c, 2c+1;   */
/*     a0*b0 rounded to binary64 first);                                  */
/*  3. the block value is a fixed pairwise tree over its 16 row values     */
/*     (rows 2m + 2m+1, then pairs of those, ...);                        */
/*  4. (a, b) is the exact sum of all block values rounded once to the     */
/*     nearest binary64 (ties to even); an exact zero is +0; a non-finite  */
/*     block value makes the result NaN.                                  */
/* Steps 1-3 are here; step 4 is a correctly rounded exact sum, done by    */
/* the Python side with math.fsum.  In the reproducible CG the vector      */
/* updates are single-rounding fused multiply-adds (fma_axpy, fma_xpby).   */
/* ------------------------------------------------------------------ */
void ora_repro_blocks(int nx, int ny, int ld, const double* a, const double* b, double* out) {
  const int nbx = (nx + 1) / 2, nby = (ny + 15) / 16;
  for (int t = 0; t < nby; ++t)
    for (int c = 0; c < nbx; ++c) {
      double v[16];
      for (int m = 0; m < 16; ++m) {
        const int j = 16 * t + m, i0 = 2 * c, i1 = 2 * c + 1;
        if (j >= ny) { v[m] = 0.0; continue; }
        const double a0 = a[(size_t)j * ld + i0], b0 = b[(size_t)j * ld + i0];
        const double a1 = i1 < nx ? a[(size_t)j * ld + i1] : 0.0;
        const double b1 = i1 < nx ? b[(size_t)j * ld + i1] : 0.0;
        const double p0 = a0 * b0;
        v[m] = fma(a1, b1, p0);
      }
      for (int w = 1; w < 16; w *= 2)
        for (int m = 0; m < 16; m += 2 * w) v[m] = v[m] + v[m + w];
      out[(size_t)t * nbx + c] = v[0];
    }
}

/* y = fma(alpha, x, y) over the interior */
void ora_fma_axpy(int nx, int ny, int ld, double* y, double alpha, const double* x) {
  for (int j = 0; j < ny; ++j)
    for (int i = 0; i < nx; ++i) y[(size_t)j * ld + i] = fma(alpha, x[(size_t)j * ld + i], y[(size_t)j * ld + i]);
}

/* y = fma(beta, y, x) over the interior (y = x + beta y, one rounding) */
void ora_fma_xpby(int nx, int ny, int ld, const double* x, double beta, double* y) {
  for (int j = 0; j < ny; ++j)
    for (int i = 0; i < nx; ++i) y[(size_t)j * ld + i] = fma(beta, y[(size_t)j * ld + i], x[(size_t)j * ld + i]);
}

/* ------------------------------------------------------------------ */
/* Compensated binary32 dot product, Dot2 of Ogita, Rump & Oishi,        */
/* "Accurate sum and dot product", SIAM J. Sci. Comput. 26 (2005):       */
/* TwoProduct by an exact fused multiply-add, TwoSum by Knuth.  Returns   */
/* the unevaluated pair (s, c); the result is s + c.                     */
/* ------------------------------------------------------------------ */
static void two_sum_f(float a, float b, float* s, float* e) {
  float x = a + b;
  float z = x - a;
  *s = x;
  *e = (a - (x - z)) + (b - z);
}

void ora_dot2_f32(int nx, int ny, int ld, const float* a, const float* b, double* out_s, double* out_c) {
  float s = 0.0f, c = 0.0f;
  for (int j = 0; j < ny; ++j)
    for (int i = 0; i < nx; ++i) {
      float ai = a[(size_t)j * ld + i], bi = b[(size_t)j * ld + i];
      float h = ai * bi;
      float l = fmaf(ai, bi, -h);   /* exact low part of the product */
      float t, e;
      two_sum_f(s, h, &t, &e);
      s = t;
      c = c + (e + l);
    }
  *out_s = s; *out_c = c;
}

/* ------------------------------------------------------------------ */
/* Mixed precision: FP64 iterative refinement around a low-precision     */
/* inner CG.  Inner storage: 1 = binary32 everywhere; 2 = bf16 p and r,   */
/* binary32 d and z.  Inner arithmetic is binary32; inner dots are Dot2;  */
/* inner scalars (alpha, beta) are formed in binary64 and rounded to      */
/* binary32 for the vector updates.  Inner variant: classic CG (Alg. 1).  */
/* With bf16 p, r the inner beta takes the Polak-Ribiere form             */
/* (r_new, r_new - r_old) / (r_old, r_old): equal to Algorithm 1's        */
/* (r_new, r_new) / (r_old, r_old) in exact arithmetic, where consecutive */
/* residuals are orthogonal, but it discounts the part of r_new that the  */
/* bf16 rounding left along r_old (without it the stored residual stalls  */
/* near 3e-2 of its start at 4096^2 and then grows).                      */
/* ------------------------------------------------------------------ */
static float stor(float v, int bf) { return bf ? bf16_to_f32(f32_to_bf16(v)) : v; }

static double dot2_pair(int nx, int ny, int ld, const float* a, const float* b) {
  double s, c; ora_dot2_f32(nx, ny, ld, a, b, &s, &c); return s + c;
}

/* Inner classic CG on A d = rin from d = 0; returns iterations used. */
static int inner_cg_f32(int nx, int ny, int ld, const float* rin, float* d, double tol_in, int maxit_in,
                        int bf, float* r, float* p, float* z, float* rp, int* brk) {
  size_t n = (size_t)ny * ld;
  memset(d, 0, n * sizeof(float));
  for (size_t t = 0; t < n; ++t) { r[t] = stor(rin[t], bf); p[t] = r[t]; }
  double g = dot2_pair(nx, ny, ld, r, r);
  double thr = tol_in * tol_in * g;
  int k = 0;
  *brk = 0;
  while (k < maxit_in && g > thr) {
    ora_lap5_apply_f32(nx, ny, ld, p, z);
    double pz = dot2_pair(nx, ny, ld, p, z);
    if (!(pz > 0.0) || !isfinite(pz)) { *brk = 1; break; }
    float a = (float)(g / pz);
    if (bf) memcpy(rp, r, n * sizeof(float));        /* r_old, for the Polak-Ribiere beta */
    for (int j = 0; j < ny; ++j)
      for (int i = 0; i < nx; ++i) {
        size_t t = (size_t)j * ld + i;
        d[t] = d[t] + a * p[t];
        r[t] = stor(r[t] - a * z[t], bf);
      }
    double gn = dot2_pair(nx, ny, ld, r, r);
    ++k;
    if (!isfinite(gn)) { *brk = 1; break; }
    double num = bf ? gn - dot2_pair(nx, ny, ld, r, rp) : gn;
    float bt = (float)(num / g);
    g = gn;
    if (g <= thr) break;
    for (int j = 0; j < ny; ++j)
      for (int i = 0; i < nx; ++i) {
        size_t t = (size_t)j * ld + i;
        p[t] = stor(r[t] + bt * p[t], bf);
      }
  }
  return k;
}

/* The inner solve alone, for the tests' pins: classic CG (Algorithm 1) on
 * A d = rin from d = 0 with the inner storage above.  On return d holds the
 * correction, r_out (may be NULL) the final stored inner residual, and
 * *breakdown is 1 if (p, Ap) <= 0 or a dot was non-finite.  Returns the
 * iterations done. */
int ora_inner_cg_f32(int nx, int ny, int ld, const float* rin, float* d, double tol_in, int maxit_in,
                     int inner_storage, float* r_out, int* breakdown) {
  const size_t n = (size_t)ny * ld;
  float *r = calloc(n, 4), *p = calloc(n, 4), *z = calloc(n, 4), *rp = calloc(n, 4);
  int brk = 0, k = -1;
  if (r && p && z && rp && (inner_storage == 1 || inner_storage == 2) && maxit_in >= 0) {
    k = inner_cg_f32(nx, ny, ld, rin, d, tol_in, maxit_in, inner_storage == 2, r, p, z, rp, &brk);
    if (r_out) memcpy(r_out, r, n * sizeof(float));
  }
  free(r); free(p); free(z); free(rp);
  if (breakdown) *breakdown = brk;
  return k;
}

/* Acceptance of a refinement step x <- x + d whose FP64 residual r_new =
 * b - A(x + d) is not below the previous one r_old (rr_new >= rr_old).  The
 * error e = A^-1 r_old has energy E = (e, A e); the step changes it by
 *   E_old - E_new = 2 (d, r_old) - (d, A d) = (d, r_old) + (d, r_new)
 * (A d = r_old - r_new).  The step is kept when (d, r_old) > 0 and it removed
 * at least half of that: (d, r_new) >= -(d, r_old) / 2 -- for d = s e this
 * holds for 0 < s <= 3/2.  An inner binary32 solve whose right-hand side is
 * dominated by the smoothest modes (kappa * u32 near 0.1) can return such a
 * d: A-norm-accurate, but with a rough residual error larger than r_old in the
 * 2-norm; the next inner solve removes the rough part quickly.  Steps that do
 * neither (d mostly rounding noise: (d, A d) dominates) are undone.
 * dro = (d, r_old), drn = (d, r_new).  Returns 1 to keep the step. */
int ora_ir_keep_step(double rr_new, double rr_old, double dro, double drn) {
  if (rr_new < rr_old) return 1;
  return dro > 0.0 && drn >= -0.5 * dro;
}

/* (d, r) with d binary32, r binary64: binary64 products and sums in index
 * order */
static double dot_fd(int nx, int ny, int ld, const float* d, const double* r) {
  double s = 0.0;
  for (int j = 0; j < ny; ++j)
    for (int i = 0; i < nx; ++i) s += (double)d[(size_t)j * ld + i] * r[(size_t)j * ld + i];
  return s;
}

int ora_cg_ir(int nx, int ny, int ld, const double* b, double* x, double tol, int max_outer,
              int inner_storage, double tol_in, int maxit_in, ora_info* info) {
  ora_info inf; memset(&inf, 0, sizeof inf);
  if (!arg_ok(nx, ny, ld, max_outer) || !b || !x || (inner_storage != 1 && inner_storage != 2) || maxit_in < 1) {
    inf.status = ORA_ERR_INVALID_ARG; if (info) *info = inf; return inf.status;
  }
  const size_t n = (size_t)ny * ld;
  double bb = ora_dot_f64(nx, ny, ld, b, b);
  if (!isfinite(bb)) { inf.status = ORA_ERR_NONFINITE; inf.relres_recursive = NAN; inf.relres_true = NAN; if (info) *info = inf; return inf.status; }
  if (bb == 0.0) { zero64(nx, ny, ld, x); inf.status = ORA_OK; if (info) *info = inf; return inf.status; }
  const double thr = tol > 0.0 ? tol * tol * bb : 0.0;
  const int bf = inner_storage == 2;
  double* r = calloc(n, 8);
  float *rin = calloc(n, 4), *d = calloc(n, 4), *ri = calloc(n, 4), *pi = calloc(n, 4), *zi = calloc(n, 4),
        *rp = calloc(n, 4);
  if (!r || !rin || !d || !ri || !pi || !zi || !rp) { free(r); free(rin); free(d); free(ri); free(pi); free(zi); free(rp); inf.status = ORA_ERR_INVALID_ARG; if (info) *info = inf; return inf.status; }
  int status = ORA_NOT_CONVERGED, outer = 0, total_inner = 0;
  double rr = 0.0, rr_prev = 0.0, dro = 0.0;
  for (;;) {
    residual64(nx, ny, ld, b, x, r);                    /* FP64 residual */
    rr = ora_dot_f64(nx, ny, ld, r, r);
    if (!isfinite(rr)) { status = ORA_ERR_NONFINITE; break; }
    if (rr <= thr) { status = ORA_OK; break; }
    if (outer > 0 && !ora_ir_keep_step(rr, rr_prev, dro, rr < rr_prev ? 0.0 : dot_fd(nx, ny, ld, d, r))) {
      /* stagnation guard: the last correction lowered neither the FP64
         residual nor, by half of what it claims, the error's energy (the
         inner precision cannot resolve this system); undo it and stop */
      for (int j = 0; j < ny; ++j)
        for (int i = 0; i < nx; ++i) x[(size_t)j * ld + i] = x[(size_t)j * ld + i] - (double)d[(size_t)j * ld + i];
      residual64(nx, ny, ld, b, x, r);
      rr = ora_dot_f64(nx, ny, ld, r, r);
      break;
    }
    rr_prev = rr;
    if (outer >= max_outer) break;
    for (size_t t = 0; t < n; ++t) rin[t] = (float)r[t]; /* round to nearest */
    int brk = 0;
    total_inner += inner_cg_f32(nx, ny, ld, rin, d, tol_in, maxit_in, bf, ri, pi, zi, rp, &brk);
    if (brk) { status = ORA_ERR_BREAKDOWN; break; }
    dro = dot_fd(nx, ny, ld, d, r);                     /* (d, r_old) */
    for (int j = 0; j < ny; ++j)                        /* FP64 update */
      for (int i = 0; i < nx; ++i) x[(size_t)j * ld + i] = x[(size_t)j * ld + i] + (double)d[(size_t)j * ld + i];
    ++outer;
  }
  inf.status = status; inf.iters = total_inner; inf.outer_iters = outer;
  inf.relres_recursive = sqrt(rr / bb);
  inf.relres_true = true_relres(nx, ny, ld, b, x, bb);
  free(r); free(rin); free(d); free(ri); free(pi); free(zi); free(rp);
  if (info) *info = inf;
  return status;
}

/* ------------------------------------------------------------------ */
/* Preconditioned CG with a geometric multigrid V-cycle as M^-1.  Not in  */
/* the paper: the preconditioned form of the cited pipelined CG (Ghysels  */
/* and Vanroose, with a general M; the paper fixes M = I).  Readings:     */
/*  - levels: grid (nx, ny) -> ((nx-1)/2, (ny-1)/2), coarse point (I, J)   */
/*    at fine (2I+1, 2J+1) (0-based); coarsening stops when either side    */
/*    of the next grid would be 0, or after max_levels grids;             */
/*  - every level's operator is the same 5-point mask (Sec. II-B): with    */
/*    the unscaled mask A_h = h^2 L_h the coarse-grid correction is        */
/*    e = P A_c^-1 P^T r, P bilinear interpolation, restriction P^T       */
/*    (weights [1 2 1; 2 4 2; 1 2 1] / 4); coarse points outside the       */
/*    coarse grid count as 0;                                              */
/*  - smoother: damped Jacobi x <- x + c (b - A x), c = omega / 4 with     */
/*    omega = 4/5 (c = 0.2), nu sweeps before and nu after the coarse      */
/*    correction (symmetric, so M is symmetric positive definite);         */
/*  - coarsest grid: nu_c damped Jacobi sweeps from 0;                     */
/*  - PCG (Algorithm 1 with M): z = M^-1 r, gamma = (r, z), p = z + beta p,*/
/*    stop when (r, r) <= tol^2 (b, b) as in the unpreconditioned solve.   */
/* Fixed operation orders (the GPU kernels follow them):                   */
/*    Jacobi:   x + c * (b - A x)                                          */
/*    restrict: 0.25 * ((4 rC + 2 ((rW + rE) + rS + rN))                   */
/*                      + ((rSW + rSE) + rNW + rNE))                        */
/*    prolong:  odd-odd e; even-odd 0.5 (eW + eE); odd-even 0.5 (eS + eN); */
/*              even-even 0.25 ((eSW + eSE) + (eNW + eNE))                 */
/* ------------------------------------------------------------------ */
#define ORA_MG_C 0.2

static double mg_at(const double* v, int nx, int ny, int i, int j) {
  return (i < 0 || i >= nx || j < 0 || j >= ny) ? 0.0 : v[(size_t)j * nx + i];
}

/* y = A x on a dense (pitch = nx) level grid, fixed add order */
static void mg_apply(int nx, int ny, const double* x, double* y) {
  for (int j = 0; j < ny; ++j)
    for (int i = 0; i < nx; ++i) {
      double acc = 4.0 * x[(size_t)j * nx + i];
      acc -= mg_at(x, nx, ny, i - 1, j);
      acc -= mg_at(x, nx, ny, i + 1, j);
      acc -= mg_at(x, nx, ny, i, j - 1);
      acc -= mg_at(x, nx, ny, i, j + 1);
      y[(size_t)j * nx + i] = acc;
    }
}

/* one damped Jacobi sweep: xo = xi + c (b - A xi) */
static void mg_jacobi(int nx, int ny, const double* b, const double* xi, double* xo, double* tmp) {
  mg_apply(nx, ny, xi, tmp);
  for (size_t t = 0; t < (size_t)nx * ny; ++t) xo[t] = xi[t] + ORA_MG_C * (b[t] - tmp[t]);
}

/* bc = P^T r (fine nx x ny -> coarse (nx-1)/2 x (ny-1)/2) */
void ora_mg_restrict(int nx, int ny, const double* r, double* bc) {
  const int nxc = (nx - 1) / 2, nyc = (ny - 1) / 2;
  for (int J = 0; J < nyc; ++J)
    for (int I = 0; I < nxc; ++I) {
      const int i = 2 * I + 1, j = 2 * J + 1;
      const double rC = mg_at(r, nx, ny, i, j);
      const double s1 = ((mg_at(r, nx, ny, i - 1, j) + mg_at(r, nx, ny, i + 1, j)) + mg_at(r, nx, ny, i, j - 1)) +
                        mg_at(r, nx, ny, i, j + 1);
      const double s2 = ((mg_at(r, nx, ny, i - 1, j - 1) + mg_at(r, nx, ny, i + 1, j - 1)) +
                         mg_at(r, nx, ny, i - 1, j + 1)) + mg_at(r, nx, ny, i + 1, j + 1);
      bc[(size_t)J * nxc + I] = 0.25 * ((4.0 * rC + 2.0 * s1) + s2);
    }
}

/* x += P ec (coarse (nx-1)/2 x (ny-1)/2 -> fine nx x ny) */
void ora_mg_prolong_add(int nx, int ny, const double* ec, double* x) {
  const int nxc = (nx - 1) / 2, nyc = (ny - 1) / 2;
  for (int j = 0; j < ny; ++j)
    for (int i = 0; i < nx; ++i) {
      double v;
      const int I = i >> 1, J = j >> 1;  /* odd i: I = (i-1)/2; even i: neighbours I-1, I */
      if ((i & 1) && (j & 1)) {
        v = mg_at(ec, nxc, nyc, I, J);
      } else if (!(i & 1) && (j & 1)) {
        v = 0.5 * (mg_at(ec, nxc, nyc, I - 1, J) + mg_at(ec, nxc, nyc, I, J));
      } else if ((i & 1) && !(j & 1)) {
        v = 0.5 * (mg_at(ec, nxc, nyc, I, J - 1) + mg_at(ec, nxc, nyc, I, J));
      } else {
        v = 0.25 * ((mg_at(ec, nxc, nyc, I - 1, J - 1) + mg_at(ec, nxc, nyc, I, J - 1)) +
                    (mg_at(ec, nxc, nyc, I - 1, J) + mg_at(ec, nxc, nyc, I, J)));
      }
      x[(size_t)j * nx + i] += v;
    }
}

/* x = V-cycle(b) from x = 0 on a dense level grid; returns 0, -1 on allocation failure */
static int mg_vcycle(int nx, int ny, const double* b, double* x, int nu, int nu_c, int levels_left) {
  const size_t n = (size_t)nx * ny;
  const int nxc = (nx - 1) / 2, nyc = (ny - 1) / 2;
  double* t = (double*)malloc(n * sizeof(double));
  double* w = (double*)malloc(n * sizeof(double));
  if (!t || !w) { free(t); free(w); return -1; }
  memset(x, 0, n * sizeof(double));
  if (nxc < 1 || nyc < 1 || levels_left <= 1) {          /* coarsest grid */
    for (int s = 0; s < nu_c; ++s) { mg_jacobi(nx, ny, b, x, w, t); memcpy(x, w, n * sizeof(double)); }
    free(t); free(w);
    return 0;
  }
  for (int s = 0; s < nu; ++s) { mg_jacobi(nx, ny, b, x, w, t); memcpy(x, w, n * sizeof(double)); }
  mg_apply(nx, ny, x, t);
  for (size_t k = 0; k < n; ++k) w[k] = b[k] - t[k];      /* residual */
  const size_t nc = (size_t)nxc * nyc;
  double* bc = (double*)malloc(nc * sizeof(double));
  double* ec = (double*)malloc(nc * sizeof(double));
  if (!bc || !ec) { free(t); free(w); free(bc); free(ec); return -1; }
  ora_mg_restrict(nx, ny, w, bc);
  int rc = mg_vcycle(nxc, nyc, bc, ec, nu, nu_c, levels_left - 1);
  if (rc == 0) {
    ora_mg_prolong_add(nx, ny, ec, x);
    for (int s = 0; s < nu; ++s) { mg_jacobi(nx, ny, b, x, w, t); memcpy(x, w, n * sizeof(double)); }
  }
  free(t); free(w); free(bc); free(ec);
  return rc;
}

/* z = M^-1 r on a pitched grid (one V-cycle; levels = 0 gives z = r) */
int ora_mg_precond(int nx, int ny, int ld, const double* r, double* z, int levels, int nu, int nu_c) {
  if (nx < 1 || ny < 1 || ld < nx || levels < 0 || nu < 0 || nu_c < 0) return ORA_ERR_INVALID_ARG;
  if (levels == 0) { copy64(nx, ny, ld, z, r); return ORA_OK; }
  const size_t n = (size_t)nx * ny;
  double* b = (double*)malloc(n * sizeof(double));
  double* x = (double*)malloc(n * sizeof(double));
  if (!b || !x) { free(b); free(x); return ORA_ERR_INVALID_ARG; }
  for (int j = 0; j < ny; ++j) memcpy(b + (size_t)j * nx, r + (size_t)j * ld, (size_t)nx * sizeof(double));
  int rc = mg_vcycle(nx, ny, b, x, nu, nu_c, levels);
  if (rc == 0)
    for (int j = 0; j < ny; ++j) memcpy(z + (size_t)j * ld, x + (size_t)j * nx, (size_t)nx * sizeof(double));
  free(b); free(x);
  return rc == 0 ? ORA_OK : ORA_ERR_INVALID_ARG;
}

int ora_cg_pcg(int nx, int ny, int ld, const double* b, double* x, double tol, int maxit, int levels, int nu,
               int nu_c, double* relres_hist, ora_info* info) {
  ora_info inf; memset(&inf, 0, sizeof inf);
  if (!arg_ok(nx, ny, ld, maxit) || !b || !x || levels < 0 || nu < 0 || nu_c < 0) {
    inf.status = ORA_ERR_INVALID_ARG; if (info) *info = inf; return inf.status;
  }
  const size_t n = (size_t)ny * ld;
  double bb = ora_dot_f64(nx, ny, ld, b, b);
  if (!isfinite(bb)) { inf.status = ORA_ERR_NONFINITE; inf.relres_recursive = NAN; inf.relres_true = NAN; if (info) *info = inf; return inf.status; }
  if (bb == 0.0) { zero64(nx, ny, ld, x); inf.status = ORA_OK; if (info) *info = inf; return inf.status; }
  const double thr = tol > 0.0 ? tol * tol * bb : 0.0;
  double *r = calloc(n, 8), *z = calloc(n, 8), *p = calloc(n, 8), *q = calloc(n, 8);
  if (!r || !z || !p || !q) { free(r); free(z); free(p); free(q); inf.status = ORA_ERR_INVALID_ARG; if (info) *info = inf; return inf.status; }
  int status = ORA_NOT_CONVERGED, k = 0;
  residual64(nx, ny, ld, b, x, r);                       /* r = b - A x0 */
  double rr = ora_dot_f64(nx, ny, ld, r, r);
  if (relres_hist) relres_hist[0] = sqrt(rr / bb);
  if (!isfinite(rr)) status = ORA_ERR_NONFINITE;
  else if (rr <= thr) status = ORA_OK;
  double gamma = 0.0;
  if (status == ORA_NOT_CONVERGED) {
    if (ora_mg_precond(nx, ny, ld, r, z, levels, nu, nu_c) != ORA_OK) status = ORA_ERR_INVALID_ARG;
    copy64(nx, ny, ld, p, z);                            /* p = z */
    gamma = ora_dot_f64(nx, ny, ld, r, z);               /* (r, z) */
    if (!(gamma > 0.0) || !isfinite(gamma)) status = ORA_ERR_BREAKDOWN;
  }
  while (status == ORA_NOT_CONVERGED && k < maxit) {
    ora_lap5_apply_f64(nx, ny, ld, p, q);                /* q = A p */
    double pq = ora_dot_f64(nx, ny, ld, p, q);
    if (!(pq > 0.0) || !isfinite(pq)) { status = ORA_ERR_BREAKDOWN; break; }
    double alpha = gamma / pq;
    axpy64(nx, ny, ld, x, alpha, p);                     /* x = x + alpha p */
    axpy64(nx, ny, ld, r, -alpha, q);                    /* r = r - alpha q */
    ++k;
    rr = ora_dot_f64(nx, ny, ld, r, r);
    if (relres_hist) relres_hist[k] = sqrt(rr / bb);
    if (!isfinite(rr)) { status = ORA_ERR_NONFINITE; break; }
    if (rr <= thr) { status = ORA_OK; break; }
    if (ora_mg_precond(nx, ny, ld, r, z, levels, nu, nu_c) != ORA_OK) { status = ORA_ERR_INVALID_ARG; break; }
    double gnew = ora_dot_f64(nx, ny, ld, r, z);         /* (r, z) */
    if (!(gnew > 0.0) || !isfinite(gnew)) { status = ORA_ERR_BREAKDOWN; break; }
    double beta = gnew / gamma;
    gamma = gnew;
    xpby64(nx, ny, ld, z, beta, p);                      /* p = z + beta p */
  }
  inf.status = status; inf.iters = k;
  inf.relres_recursive = sqrt(rr / bb);
  inf.relres_true = true_relres(nx, ny, ld, b, x, bb);
  free(r); free(z); free(p); free(q);
  if (info) *info = inf;
  return status;
}

/* ------------------------------------------------------------------ */
/* Pipelined preconditioned CG: Algorithm 2 with a preconditioner, in the  */
/* general form of the cited Ghysels-Vanroose method (the paper fixes     */
/* M = I, where u = r, m = w and s = q below and the recurrences reduce to */
/* Algorithm 2 line by line).  With M^-1 the multigrid V-cycle above:     */
/*   r = b - A x, u = M^-1 r, w = A u;                                     */
/*   per iteration: gamma = (r, u), delta = (w, u), m = M^-1 w, n = A m;   */
/*   beta = gamma / gamma_old, alpha = 1 / (delta / gamma - beta / alpha)  */
/*   (first: beta = 0, alpha = gamma / delta);                             */
/*   z = n + beta z, q = m + beta q, s = w + beta s, p = u + beta p;       */
/*   x += alpha p, r -= alpha s, u -= alpha q, w -= alpha z.               */
/* Stops when (r, r) <= tol^2 (b, b), tested where gamma is formed.        */
/* ------------------------------------------------------------------ */
int ora_cg_ppcg(int nx, int ny, int ld, const double* b, double* x, double tol, int maxit, int levels, int nu,
                int nu_c, ora_info* info) {
  ora_info inf; memset(&inf, 0, sizeof inf);
  if (!arg_ok(nx, ny, ld, maxit) || !b || !x || levels < 0 || nu < 0 || nu_c < 0) {
    inf.status = ORA_ERR_INVALID_ARG; if (info) *info = inf; return inf.status;
  }
  const size_t n = (size_t)ny * ld;
  double bb = ora_dot_f64(nx, ny, ld, b, b);
  if (!isfinite(bb)) { inf.status = ORA_ERR_NONFINITE; inf.relres_recursive = NAN; inf.relres_true = NAN; if (info) *info = inf; return inf.status; }
  if (bb == 0.0) { zero64(nx, ny, ld, x); inf.status = ORA_OK; if (info) *info = inf; return inf.status; }
  const double thr = tol > 0.0 ? tol * tol * bb : 0.0;
  double *r = calloc(n, 8), *u = calloc(n, 8), *w = calloc(n, 8), *m = calloc(n, 8), *nv = calloc(n, 8);
  double *z = calloc(n, 8), *q = calloc(n, 8), *s = calloc(n, 8), *p = calloc(n, 8);
  if (!r || !u || !w || !m || !nv || !z || !q || !s || !p) {
    free(r); free(u); free(w); free(m); free(nv); free(z); free(q); free(s); free(p);
    inf.status = ORA_ERR_INVALID_ARG; if (info) *info = inf; return inf.status;
  }
  int status = ORA_NOT_CONVERGED, k = 0;
  double rr = 0.0, gamma = 0.0, alpha = 0.0;
  residual64(nx, ny, ld, b, x, r);                       /* r = b - A x */
  if (ora_mg_precond(nx, ny, ld, r, u, levels, nu, nu_c) != ORA_OK) status = ORA_ERR_INVALID_ARG;
  ora_lap5_apply_f64(nx, ny, ld, u, w);                  /* w = A u */
  while (status == ORA_NOT_CONVERGED) {
    const double gamma_old = gamma;
    rr = ora_dot_f64(nx, ny, ld, r, r);
    if (!isfinite(rr)) { status = ORA_ERR_NONFINITE; break; }
    if (rr <= thr) { status = ORA_OK; break; }
    if (k >= maxit) break;
    gamma = ora_dot_f64(nx, ny, ld, r, u);               /* gamma = (r, u) */
    const double delta = ora_dot_f64(nx, ny, ld, w, u);  /* delta = (w, u) */
    if (ora_mg_precond(nx, ny, ld, w, m, levels, nu, nu_c) != ORA_OK) { status = ORA_ERR_INVALID_ARG; break; }
    ora_lap5_apply_f64(nx, ny, ld, m, nv);               /* n = A m */
    double beta;
    if (k == 0) {
      if (!(delta > 0.0) || !isfinite(delta) || !(gamma > 0.0)) { status = ORA_ERR_BREAKDOWN; break; }
      beta = 0.0;
      alpha = gamma / delta;
      copy64(nx, ny, ld, z, nv);                         /* z = n, q = m, s = w, p = u */
      copy64(nx, ny, ld, q, m);
      copy64(nx, ny, ld, s, w);
      copy64(nx, ny, ld, p, u);
    } else {
      beta = gamma / gamma_old;
      const double denom = delta / gamma - beta / alpha;
      if (!(denom > 0.0) || !isfinite(denom) || !(gamma > 0.0)) { status = ORA_ERR_BREAKDOWN; break; }
      alpha = 1.0 / denom;
      xpby64(nx, ny, ld, nv, beta, z);                   /* z = n + beta z */
      xpby64(nx, ny, ld, m, beta, q);                    /* q = m + beta q */
      xpby64(nx, ny, ld, w, beta, s);                    /* s = w + beta s */
      xpby64(nx, ny, ld, u, beta, p);                    /* p = u + beta p */
    }
    axpy64(nx, ny, ld, x, alpha, p);                     /* x = x + alpha p */
    axpy64(nx, ny, ld, r, -alpha, s);                    /* r = r - alpha s */
    axpy64(nx, ny, ld, u, -alpha, q);                    /* u = u - alpha q */
    axpy64(nx, ny, ld, w, -alpha, z);                    /* w = w - alpha z */
    ++k;
  }
  inf.status = status; inf.iters = k;
  inf.relres_recursive = sqrt(rr / bb);
  inf.relres_true = true_relres(nx, ny, ld, b, x, bb);
  free(r); free(u); free(w); free(m); free(nv); free(z); free(q); free(s); free(p);
  if (info) *info = inf;
  return status;
}
