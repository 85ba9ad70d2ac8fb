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
                       residual replacement.
  cg_ir             -- FP64 iterative refinement around a binary32 (or bf16
                       p/r) inner Algorithm 1 with Dot2 inner dot products.
  dot2_f32          -- Dot2 (Ogita, Rump & Oishi 2005).
"""
import ctypes
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
        path = _build.build()
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
        L.ora_cg_ir.argtypes = [i, i, i, vp, vp, d, i, i, d, i, ctypes.POINTER(Info)]
        for name in ("ora_cg_classic", "ora_cg_newcg", "ora_cg_ir"):
            getattr(L, name).restype = i
        L.ora_f32_to_bf16.argtypes = [ctypes.c_float]
        L.ora_f32_to_bf16.restype = ctypes.c_uint16
        _lib = L
    return _lib


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


def cg_newcg(b, x0=None, tol=1e-10, maxit=1000, nx=None, rr_period=0, trace=None):
    """Algorithm 2 (de-garbled).  Returns (x, info dict)."""
    ny, ld = b.shape
    nx = ld if nx is None else nx
    b = _grid(b, np.float64, nx)
    x = np.zeros_like(b) if x0 is None else _grid(x0, np.float64, nx).copy()
    info = Info()
    lib().ora_cg_newcg(nx, ny, ld, _ptr(b), _ptr(x), tol, maxit, rr_period,
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
    if maxit_in is None:
        maxit_in = 4 * (nx + ny) + 50
    info = Info()
    lib().ora_cg_ir(nx, ny, ld, _ptr(b), _ptr(x), tol, max_outer, storage, tol_in, maxit_in, ctypes.byref(info))
    return x, info.as_dict()


def cg_solve(b, variant="classic", **kw):
    if variant == "classic":
        return cg_classic(b, **kw)
    if variant == "newcg":
        return cg_newcg(b, **kw)
    raise ValueError(variant)
