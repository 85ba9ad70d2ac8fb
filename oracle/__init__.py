"""CPU oracle for matrix-free CG on the 2D Dirichlet 5-point Laplacian.

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg are the only users.  The product path (the CUDA
library and its binding) never imports this package, and this package never
imports the product.

Everything here is a thin ctypes marshalling layer over ``lap5_oracle.c``
(plain C, binary64 unless a function says otherwise).  Arrays are numpy arrays
of shape (ny, ld) with ld >= nx; only the first nx columns are the grid.

Functions and the passages they follow (arxiv 1803.03797):
  lap5_apply        -- Sec. II-B, the 3x3 mask [0 -1 0; -1 4 -1; 0 -1 0] with
                       zero Dirichlet boundary (Sec. II problem statement).
  cg_classic        -- Algorithm 1 (stdCG), x0 allowed.
  cg_newcg          -- Algorithm 2 (NewCG), de-garbled after the cited
                       Ghysels-Vanroose pipelined CG with M = I; optional
                       residual replacement; optional alpha from dot
                       products of the current vectors (stable=True).
  cg_ir             -- FP64 iterative refinement around a binary32 (or bf16
                       p/r) inner Algorithm 1 with Dot2 inner dot products.
  inner_cg_f32      -- that inner solve alone (for its own pins).
  dot2_f32          -- Dot2 (Ogita, Rump & Oishi 2005).
  mg_precond, cg_pcg -- preconditioned CG (Algorithm 1 with M) with a
                       geometric multigrid V-cycle as M^-1 (the cited
                       pipelined CG's general form; the paper fixes M = I).
  dot_repro, cg_classic_repro, cg_newcg_repro
                    -- the reproducible mode: a dot product whose value does
                       not depend on how the work is split (the paper
                       accumulates in fixed point because floating-point
                       addition is not associative, Sec. III; the dot product
                       is a multiplier-adder tree, Sec. II-C-1), and
                       Algorithms 1 / 2 with those dots and single-rounding
                       vector updates.
"""
import ctypes
import math
import numpy as np

from . import build as _build

OK, NOT_CONVERGED, ERR_INVALID_ARG, ERR_BREAKDOWN, ERR_NONFINITE = 0, 1, -1, -3, -5

_lib = None


class Info(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("iters", ctypes.c_int32),
                ("outer_iters", ctypes.c_int32), ("pad", ctypes.c_int32),
                ("relres_recursive", ctypes.c_double), ("relres_true", ctypes.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_ if k != "pad"}


class _Trace(ctypes.Structure):
    _fields_ = [(n, ctypes.c_void_p) for n in ("x", "r", "p", "w", "q", "z", "alpha", "beta", "relres")] + [
        ("ntrace", ctypes.c_int32), ("pad", ctypes.c_int32)]


def lib():
    global _lib
    if _lib is None:
        _lib = _load(_build.build())
    return _lib


_lib_omp = None


class timing_build:
    """Context manager: inside it, every oracle function runs the OpenMP timing
    build of lap5_oracle.c (its binary64 row loops on all threads, dot products
    as per-thread partial sums added in thread order).  For the benchmark's
    CPU-baseline timing only; parity always uses the sequential build.
    ``threads`` is the number of threads that build uses."""

    def __enter__(self):
        global _lib, _lib_omp
        if _lib_omp is None:
            _lib_omp = _load(_build.build(openmp=True))
        self.saved = _lib
        _lib = _lib_omp
        self.threads = int(_lib_omp.ora_threads())
        return self

    def __exit__(self, *exc):
        global _lib
        _lib = self.saved
        return False


def _load(path):
    L = ctypes.CDLL(path)
    i, d, vp = ctypes.c_int, ctypes.c_double, ctypes.c_void_p
    for name in ("ora_lap5_apply_f64", "ora_lap5_apply_f32", "ora_lap5_apply_bf16"):
        getattr(L, name).argtypes = [i, i, i, vp, vp]
        getattr(L, name).restype = None
    L.ora_dot_f64.argtypes = [i, i, i, vp, vp]
    L.ora_dot_f64.restype = d
    L.ora_dot2_f32.argtypes = [i, i, i, vp, vp, ctypes.POINTER(d), ctypes.POINTER(d)]
    L.ora_dot2_f32.restype = None
    L.ora_cg_classic.argtypes = [i, i, i, vp, vp, d, i, ctypes.POINTER(_Trace), ctypes.POINTER(Info)]
    L.ora_cg_newcg.argtypes = [i, i, i, vp, vp, d, i, i, ctypes.POINTER(_Trace), ctypes.POINTER(Info)]
    L.ora_cg_newcg_stable.argtypes = [i, i, i, vp, vp, d, i, i, ctypes.POINTER(_Trace), ctypes.POINTER(Info)]
    L.ora_cg_newcg_stable.restype = i
    L.ora_cg_ir.argtypes = [i, i, i, vp, vp, d, i, i, d, i, ctypes.POINTER(Info)]
    L.ora_inner_cg_f32.argtypes = [i, i, i, vp, vp, d, i, i, vp, ctypes.POINTER(i)]
    L.ora_inner_cg_f32.restype = i
    L.ora_ir_keep_step.argtypes = [d, d, d, d]
    L.ora_ir_keep_step.restype = i
    for name in ("ora_cg_classic", "ora_cg_newcg", "ora_cg_ir"):
        getattr(L, name).restype = i
    L.ora_repro_blocks.argtypes = [i, i, i, vp, vp, vp]
    L.ora_repro_blocks.restype = None
    L.ora_fma_axpy.argtypes = [i, i, i, vp, d, vp]
    L.ora_fma_axpy.restype = None
    L.ora_fma_xpby.argtypes = [i, i, i, vp, d, vp]
    L.ora_fma_xpby.restype = None
    L.ora_mg_restrict.argtypes = [i, i, vp, vp]
    L.ora_mg_restrict.restype = None
    L.ora_mg_prolong_add.argtypes = [i, i, vp, vp]
    L.ora_mg_prolong_add.restype = None
    L.ora_mg_precond.argtypes = [i, i, i, vp, vp, i, i, i]
    L.ora_mg_precond.restype = i
    L.ora_cg_pcg.argtypes = [i, i, i, vp, vp, d, i, i, i, i, vp, ctypes.POINTER(Info)]
    L.ora_cg_pcg.restype = i
    L.ora_cg_ppcg.argtypes = [i, i, i, vp, vp, d, i, i, i, i, ctypes.POINTER(Info)]
    L.ora_cg_ppcg.restype = i
    L.ora_f32_to_bf16.argtypes = [ctypes.c_float]
    L.ora_f32_to_bf16.restype = ctypes.c_uint16
    L.ora_threads.argtypes = []
    L.ora_threads.restype = i
    return L


def _grid(a, dtype, nx):
    a = np.ascontiguousarray(a, dtype=dtype)
    if a.ndim != 2 or a.shape[1] < nx:
        raise ValueError("expected a (ny, ld) array with ld >= nx")
    return a


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p) if a is not None else None


def lap5_apply(x, nx=None, dtype=np.float64):
    """y = A x for the 5-point Dirichlet Laplacian (Sec. II-B mask).

    dtype float64 / float32: arithmetic in that precision with the fixed add
    order 4*xC - xW - xE - xS - xN.  dtype 'bf16': x holds bf16 bit patterns
    (uint16); arithmetic is binary32 and the result is rounded to bf16.
    Padding columns of y are zero."""
    ny, ld = x.shape
    nx = ld if nx is None else nx
    if dtype == "bf16":
        x = _grid(x, np.uint16, nx)
        y = np.zeros_like(x)
        lib().ora_lap5_apply_bf16(nx, ny, ld, _ptr(x), _ptr(y))
        return y
    x = _grid(x, dtype, nx)
    y = np.zeros_like(x)
    fn = lib().ora_lap5_apply_f64 if x.dtype == np.float64 else lib().ora_lap5_apply_f32
    fn(nx, ny, ld, _ptr(x), _ptr(y))
    return y


def dot(a, b, nx=None):
    ny, ld = a.shape
    nx = ld if nx is None else nx
    a = _grid(a, np.float64, nx)
    b = _grid(b, np.float64, nx)
    return lib().ora_dot_f64(nx, ny, ld, _ptr(a), _ptr(b))


def dot2_f32(a, b, nx=None):
    """Compensated binary32 dot product (Dot2); returns (s, c), result s + c."""
    ny, ld = a.shape
    nx = ld if nx is None else nx
    a = _grid(a, np.float32, nx)
    b = _grid(b, np.float32, nx)
    s, c = ctypes.c_double(), ctypes.c_double()
    lib().ora_dot2_f32(nx, ny, ld, _ptr(a), _ptr(b), ctypes.byref(s), ctypes.byref(c))
    return s.value, c.value


def f32_to_bf16_bits(v):
    """Round binary32 values to bf16 (nearest, ties to even); returns uint16 bit patterns."""
    v = np.asarray(v, dtype=np.float32)
    out = np.empty(v.shape, dtype=np.uint16)
    L = lib()
    flat_in, flat_out = v.reshape(-1), out.reshape(-1)
    for k in range(flat_in.size):
        flat_out[k] = L.ora_f32_to_bf16(float(flat_in[k]))
    return out


def bf16_bits_to_f32(h):
    h = np.asarray(h, dtype=np.uint16)
    return (h.astype(np.uint32) << 16).view(np.float32)


class Trace:
    """Numpy-backed per-iteration record (see ora_trace in lap5_oracle.c)."""

    def __init__(self, ny, ld, ntrace, maxit, newcg=False):
        shape = (ntrace, ny, ld)
        self.x = np.zeros(shape)
        self.r = np.zeros(shape)
        self.p = np.zeros(shape)
        self.w = np.zeros(shape) if newcg else None
        self.q = np.zeros(shape) if newcg else None
        self.z = np.zeros(shape) if newcg else None
        self.alpha = np.full(ntrace, np.nan)
        self.beta = np.full(ntrace, np.nan)
        self.relres = np.full(maxit + 1, np.nan)
        self._c = _Trace(*[_ptr(getattr(self, n)) for n in ("x", "r", "p", "w", "q", "z", "alpha", "beta", "relres")],
                         ntrace, 0)


def cg_classic(b, x0=None, tol=1e-10, maxit=1000, nx=None, trace=None):
    """Algorithm 1.  Returns (x, info dict)."""
    ny, ld = b.shape
    nx = ld if nx is None else nx
    b = _grid(b, np.float64, nx)
    x = np.zeros_like(b) if x0 is None else _grid(x0, np.float64, nx).copy()
    info = Info()
    lib().ora_cg_classic(nx, ny, ld, _ptr(b), _ptr(x), tol, maxit,
                         ctypes.byref(trace._c) if trace is not None else None, ctypes.byref(info))
    return x, info.as_dict()


def cg_newcg(b, x0=None, tol=1e-10, maxit=1000, nx=None, rr_period=0, trace=None, stable=False):
    """Algorithm 2 (de-garbled).  stable=True forms alpha from (p, A p)
    expanded into dot products of the current vectors instead of the scalar
    recurrence.  Returns (x, info dict)."""
    ny, ld = b.shape
    nx = ld if nx is None else nx
    b = _grid(b, np.float64, nx)
    x = np.zeros_like(b) if x0 is None else _grid(x0, np.float64, nx).copy()
    info = Info()
    fn = lib().ora_cg_newcg_stable if stable else lib().ora_cg_newcg
    fn(nx, ny, ld, _ptr(b), _ptr(x), tol, maxit, rr_period,
       ctypes.byref(trace._c) if trace is not None else None, ctypes.byref(info))
    return x, info.as_dict()


def cg_ir(b, x0=None, tol=1e-10, max_outer=60, inner="f32", tol_in=None, maxit_in=None, nx=None):
    """FP64 refinement around an inner classic CG stored in binary32 ('f32') or
    with bf16 p and r ('bf16pr').  Returns (x, info dict)."""
    ny, ld = b.shape
    nx = ld if nx is None else nx
    b = _grid(b, np.float64, nx)
    x = np.zeros_like(b) if x0 is None else _grid(x0, np.float64, nx).copy()
    storage = {"f32": 1, "bf16pr": 2}[inner]
    if tol_in is None:
        tol_in = 1e-4 if inner == "f32" else 1e-2
    if maxit_in is None:  # the inner iteration cap of each refinement step
        maxit_in = 4 * (nx + ny) + 50 if inner == "f32" else 2 * (nx + ny) + 50
    info = Info()
    lib().ora_cg_ir(nx, ny, ld, _ptr(b), _ptr(x), tol, max_outer, storage, tol_in, maxit_in, ctypes.byref(info))
    return x, info.as_dict()


def inner_cg_f32(rin, tol_in=1e-4, maxit_in=1000, storage="f32", nx=None):
    """The refinement's inner solve alone: classic CG (Algorithm 1) on
    A d = rin from d = 0 in binary32 arithmetic with Dot2 dot products; p and
    r stored in binary32 ('f32') or bf16 ('bf16pr').  rin: binary32 (ny, ld).
    Returns (d, r_final, iterations, breakdown)."""
    ny, ld = rin.shape
    nx = ld if nx is None else nx
    rin = _grid(rin, np.float32, nx)
    d = np.zeros_like(rin)
    r = np.zeros_like(rin)
    brk = ctypes.c_int(0)
    k = lib().ora_inner_cg_f32(nx, ny, ld, _ptr(rin), _ptr(d), float(tol_in), int(maxit_in),
                               {"f32": 1, "bf16pr": 2}[storage], _ptr(r), ctypes.byref(brk))
    if k < 0:
        raise ValueError("invalid arguments")
    return d, r, k, bool(brk.value)


def ir_keep_step(rr_new, rr_old, d_r_old, d_r_new):
    """The refinement's acceptance rule for a step x <- x + d: True when the
    FP64 residual fell (rr_new < rr_old) or the error's energy fell by at least
    half of (d, r_old) > 0, i.e. (d, r_new) >= -(d, r_old) / 2."""
    return bool(lib().ora_ir_keep_step(float(rr_new), float(rr_old), float(d_r_old), float(d_r_new)))


def cg_solve(b, variant="classic", **kw):
    if variant == "classic":
        return cg_classic(b, **kw)
    if variant == "newcg":
        return cg_newcg(b, **kw)
    raise ValueError(variant)


# ---------------------------------------------------------------------------
# Reproducible mode.  Definition of (a, b) (steps 1-3 in lap5_oracle.c):
#   1. blocks of 2 columns x 16 rows aligned at column 2c, row 16t (points
#      outside the grid: a = b = 0);
#   2. row value fma(a1, b1, a0*b0);
#   3. block value: fixed pairwise tree over the 16 row values;
#   4. the exact sum of the block values, rounded once to nearest (ties to
#      even); exact zero -> +0; a non-finite block value -> NaN.
# Step 4 uses math.fsum, which returns the correctly rounded exact sum.
# ---------------------------------------------------------------------------
def repro_blocks(a, b, nx=None):
    """Block values of steps 1-3, shape (ceil(ny/16), ceil(nx/2))."""
    ny, ld = a.shape
    nx = ld if nx is None else nx
    a = _grid(a, np.float64, nx)
    b = _grid(b, np.float64, nx)
    out = np.empty(((ny + 15) // 16, (nx + 1) // 2))
    lib().ora_repro_blocks(nx, ny, ld, _ptr(a), _ptr(b), _ptr(out))
    return out


def exact_sum(values):
    """Correctly rounded exact sum (step 4)."""
    v = np.asarray(values, dtype=np.float64).reshape(-1)
    if not np.all(np.isfinite(v)):
        return math.nan
    try:
        s = math.fsum(v.tolist())
    except OverflowError:
        return math.nan
    return s + 0.0  # an exact zero is +0


def dot_repro(a, b, nx=None):
    return exact_sum(repro_blocks(a, b, nx))


def _fma_axpy(y, alpha, x, nx):
    ny, ld = y.shape
    lib().ora_fma_axpy(nx, ny, ld, _ptr(y), float(alpha), _ptr(x))


def _fma_xpby(x, beta, y, nx):
    ny, ld = y.shape
    lib().ora_fma_xpby(nx, ny, ld, _ptr(x), float(beta), _ptr(y))


def _apply(x, nx):
    return lap5_apply(x, nx=nx)


def _residual(b, x, nx):
    r = np.zeros_like(b)
    r[:, :nx] = b[:, :nx] - _apply(x, nx)[:, :nx]  # one rounding per element
    return r


def _finish(status, k, gamma, bb, b, x, nx):
    res = _residual(b, x, nx)
    rt = dot_repro(res, res, nx)
    return x, {"status": status, "iters": k, "outer_iters": 0, "relres_recursive": math.sqrt(gamma / bb),
               "relres_true": math.sqrt(rt / bb)}


def cg_classic_repro(b, x0=None, tol=1e-10, maxit=1000, nx=None, history=None):
    """Algorithm 1 with reproducible dot products and fused updates
    (x = fma(alpha, p, x), r = fma(-alpha, z, r), p = fma(beta, p, r)).
    history, if a list, receives sqrt(gamma_k / (b, b)) for k = 0, 1, ..."""
    ny, ld = b.shape
    nx = ld if nx is None else nx
    b = _grid(b, np.float64, nx).copy()
    b[:, nx:] = 0.0
    x = np.zeros_like(b) if x0 is None else _grid(x0, np.float64, nx).copy()
    x[:, nx:] = 0.0
    bb = dot_repro(b, b, nx)
    if not math.isfinite(bb):
        return x, {"status": ERR_NONFINITE, "iters": 0, "outer_iters": 0, "relres_recursive": math.nan,
                   "relres_true": math.nan}
    if bb == 0.0:
        x[:] = 0.0
        return x, {"status": OK, "iters": 0, "outer_iters": 0, "relres_recursive": 0.0, "relres_true": 0.0}
    thr = tol * tol * bb if tol > 0 else 0.0
    r = _residual(b, x, nx)                      # r = b - A x0
    gamma = dot_repro(r, r, nx)                  # (r, r)
    p = r.copy()                                 # p = r
    if history is not None:
        history.append(math.sqrt(gamma / bb))
    status, k = NOT_CONVERGED, 0
    if not math.isfinite(gamma):
        status = ERR_NONFINITE
    elif gamma <= thr:
        status = OK
    while status == NOT_CONVERGED and k < maxit:
        z = _apply(p, nx)                        # z = A p
        pz = dot_repro(p, z, nx)                 # (p, z)
        if not (pz > 0.0) or not math.isfinite(pz):
            status = ERR_BREAKDOWN
            break
        alpha = gamma / pz
        _fma_axpy(x, alpha, p, nx)               # x = x + alpha p
        _fma_axpy(r, -alpha, z, nx)              # r = r - alpha z
        gnew = dot_repro(r, r, nx)
        k += 1
        if history is not None:
            history.append(math.sqrt(gnew / bb))
        if not math.isfinite(gnew):
            status, gamma = ERR_NONFINITE, gnew
            break
        beta = gnew / gamma
        gamma = gnew
        if gnew <= thr:
            status = OK
            break
        _fma_xpby(r, beta, p, nx)                # p = r + beta p
    return _finish(status, k, gamma, bb, b, x, nx)


def cg_newcg_repro(b, x0=None, tol=1e-10, maxit=1000, nx=None, rr_period=0, history=None):
    """Algorithm 2 (de-garbled as cg_newcg) with reproducible dot products
    and fused updates (z = fma(beta, z, n), q = fma(beta, q, w),
    p = fma(beta, p, r), x = fma(alpha, p, x), r = fma(-alpha, q, r),
    w = fma(-alpha, z, w))."""
    ny, ld = b.shape
    nx = ld if nx is None else nx
    b = _grid(b, np.float64, nx).copy()
    b[:, nx:] = 0.0
    x = np.zeros_like(b) if x0 is None else _grid(x0, np.float64, nx).copy()
    x[:, nx:] = 0.0
    bb = dot_repro(b, b, nx)
    if not math.isfinite(bb):
        return x, {"status": ERR_NONFINITE, "iters": 0, "outer_iters": 0, "relres_recursive": math.nan,
                   "relres_true": math.nan}
    if bb == 0.0:
        x[:] = 0.0
        return x, {"status": OK, "iters": 0, "outer_iters": 0, "relres_recursive": 0.0, "relres_true": 0.0}
    thr = tol * tol * bb if tol > 0 else 0.0
    status, k = NOT_CONVERGED, 0
    r = _residual(b, x, nx)                      # r = b - A x
    w = _apply(r, nx)                            # w = A r
    gamma = dot_repro(r, r, nx)                  # gamma = (r, r)
    if history is not None:
        history.append(math.sqrt(gamma / bb))
    alpha = 0.0
    if not math.isfinite(gamma):
        status = ERR_NONFINITE
    elif gamma <= thr:
        status = OK
    elif maxit > 0:
        delta = dot_repro(w, r, nx)              # delta = (w, r)
        n = _apply(w, nx)                        # n = A w
        if not (delta > 0.0) or not math.isfinite(delta):
            status = ERR_BREAKDOWN
        else:
            alpha = gamma / delta                # alpha = gamma / delta (beta = 0)
            z, q, p = n.copy(), w.copy(), r.copy()   # z = n, q = w, p = r
            _fma_axpy(x, alpha, p, nx)           # x = x + alpha p
            _fma_axpy(r, -alpha, q, nx)          # r = r - alpha q
            _fma_axpy(w, -alpha, z, nx)          # w = w - alpha z
            k = 1
    while status == NOT_CONVERGED and k >= 1:
        if rr_period > 0 and k % rr_period == 0:  # residual replacement
            r = _residual(b, x, nx)
            w = _apply(r, nx)
            q = _apply(p, nx)
            z = _apply(q, nx)
        gamma_old = gamma                        # gamma_old = gamma
        gamma = dot_repro(r, r, nx)              # gamma = (r, r)
        if history is not None:
            history.append(math.sqrt(gamma / bb))
        if not math.isfinite(gamma):
            status = ERR_NONFINITE
            break
        if gamma <= thr:
            status = OK
            break
        if k >= maxit:
            break
        delta = dot_repro(w, r, nx)              # delta = (w, r)
        n = _apply(w, nx)                        # n = A w
        beta = gamma / gamma_old                 # beta = gamma / gamma_old
        denom = delta / gamma - beta / alpha     # de-garbled alpha update
        if not (denom > 0.0) or not math.isfinite(denom):
            status = ERR_BREAKDOWN
            break
        alpha = 1.0 / denom
        _fma_xpby(n, beta, z, nx)                # z = n + beta z
        _fma_xpby(w, beta, q, nx)                # q = w + beta q
        _fma_xpby(r, beta, p, nx)                # p = r + beta p
        _fma_axpy(x, alpha, p, nx)               # x = x + alpha p
        _fma_axpy(r, -alpha, q, nx)              # r = r - alpha q
        _fma_axpy(w, -alpha, z, nx)              # w = w - alpha z
        k += 1
    return _finish(status, k, gamma, bb, b, x, nx)


# ---------------------------------------------------------------------------
# Multigrid-preconditioned CG (readings in lap5_oracle.c).  Level grids are
# dense (pitch = nx); the solver's grids are pitched like the other solvers.
# ---------------------------------------------------------------------------
MG_LEVELS, MG_NU, MG_NU_COARSE = 30, 2, 8


def mg_coarse_shape(ny, nx):
    return (ny - 1) // 2, (nx - 1) // 2


def mg_restrict(r):
    """P^T r for a dense (ny, nx) fine grid."""
    r = np.ascontiguousarray(r, dtype=np.float64)
    ny, nx = r.shape
    out = np.zeros(mg_coarse_shape(ny, nx))
    lib().ora_mg_restrict(nx, ny, _ptr(r), _ptr(out))
    return out


def mg_prolong_add(ec, x):
    """x + P ec for a dense coarse grid ec and fine grid x (returns a copy)."""
    x = np.ascontiguousarray(x, dtype=np.float64).copy()
    ec = np.ascontiguousarray(ec, dtype=np.float64)
    ny, nx = x.shape
    assert ec.shape == mg_coarse_shape(ny, nx)
    lib().ora_mg_prolong_add(nx, ny, _ptr(ec), _ptr(x))
    return x


def mg_precond(r, nx=None, levels=MG_LEVELS, nu=MG_NU, nu_coarse=MG_NU_COARSE):
    """z = M^-1 r: one V(nu, nu) cycle from z = 0 (levels = 0: z = r)."""
    ny, ld = r.shape
    nx = ld if nx is None else nx
    r = _grid(r, np.float64, nx)
    z = np.zeros_like(r)
    rc = lib().ora_mg_precond(nx, ny, ld, _ptr(r), _ptr(z), levels, nu, nu_coarse)
    if rc != OK:
        raise RuntimeError("ora_mg_precond: %d" % rc)
    return z


def cg_pcg(b, x0=None, tol=1e-10, maxit=1000, nx=None, levels=MG_LEVELS, nu=MG_NU, nu_coarse=MG_NU_COARSE,
           history=False):
    """Algorithm 1 with M^-1 = one multigrid V-cycle.  Returns (x, info dict)
    and, with history=True, also the relative residuals after each update."""
    ny, ld = b.shape
    nx = ld if nx is None else nx
    b = _grid(b, np.float64, nx)
    x = np.zeros_like(b) if x0 is None else _grid(x0, np.float64, nx).copy()
    hist = np.full(maxit + 1, np.nan)
    info = Info()
    lib().ora_cg_pcg(nx, ny, ld, _ptr(b), _ptr(x), tol, maxit, levels, nu, nu_coarse, _ptr(hist),
                     ctypes.byref(info))
    if history:
        return x, info.as_dict(), hist[:info.iters + 1]
    return x, info.as_dict()


def cg_ppcg(b, x0=None, tol=1e-10, maxit=1000, nx=None, levels=MG_LEVELS, nu=MG_NU, nu_coarse=MG_NU_COARSE):
    """Pipelined preconditioned CG (Algorithm 2 with M^-1 = one V-cycle;
    levels = 0 gives M = I).  Returns (x, info dict)."""
    ny, ld = b.shape
    nx = ld if nx is None else nx
    b = _grid(b, np.float64, nx)
    x = np.zeros_like(b) if x0 is None else _grid(x0, np.float64, nx).copy()
    info = Info()
    lib().ora_cg_ppcg(nx, ny, ld, _ptr(b), _ptr(x), tol, maxit, levels, nu, nu_coarse, ctypes.byref(info))
    return x, info.as_dict()
