"""lap5cg: matrix-free conjugate gradient for the 2D Dirichlet 5-point
Laplacian on an NVIDIA GB300 (sm_103a), after arxiv 1803.03797
("Efficient FPGA Implementation of Conjugate Gradient Methods for Laplacian
System using HLS").

This module is a thin ctypes binding over ``liblap5cg.so`` (C ABI in
``include/lap5cg.h``).  It only marshals arguments: torch provides device
memory and the current CUDA stream; every step of every solve runs in the
library's CUDA kernels.  There is no CPU fallback: if the library is missing or
no GPU is present, calls raise.

Grids are torch tensors of shape (ny, ld) (or (nrhs, ny, ld)) with ld >= nx;
element (i, j) is ``t[j, i]``; columns nx..ld-1 are padding and never written.
"""
import ctypes
import os

import numpy as np
import torch

from . import build as _build

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "liblap5cg.so")

OK, NOT_CONVERGED = 0, 1
ERR_INVALID_ARG, ERR_CUDA, ERR_BREAKDOWN, ERR_SYNC_TIMEOUT = -1, -2, -3, -4
ERR_NONFINITE, ERR_UNSUPPORTED, ERR_WORKSPACE = -5, -6, -7

CLASSIC, NEWCG = 0, 1
PREC_F64, PREC_F32, PREC_IR_F32, PREC_IR_BF16PR, PREC_MG_F32, PREC_MG_F64 = 0, 1, 2, 3, 4, 5
DT_F64, DT_F32, DT_BF16 = 0, 1, 2
MAX_BATCH = 1024

_VARIANTS = {"classic": CLASSIC, "newcg": NEWCG, CLASSIC: CLASSIC, NEWCG: NEWCG}
_PRECISIONS = {"f64": PREC_F64, "f32": PREC_F32, "ir_f32": PREC_IR_F32, "ir_bf16pr": PREC_IR_BF16PR,
               "mg_f32": PREC_MG_F32, "mg_f64": PREC_MG_F64,
               PREC_F64: PREC_F64, PREC_F32: PREC_F32, PREC_IR_F32: PREC_IR_F32, PREC_IR_BF16PR: PREC_IR_BF16PR,
               PREC_MG_F32: PREC_MG_F32, PREC_MG_F64: PREC_MG_F64}

INFO_DTYPE = np.dtype([("status", "<i4"), ("iters", "<i4"), ("outer_iters", "<i4"), ("pad", "<i4"),
                       ("relres_recursive", "<f8"), ("relres_true", "<f8")])
INFO_BYTES = INFO_DTYPE.itemsize


class Opts(ctypes.Structure):
    """Mirror of lap5cg_opts."""
    _fields_ = [("rr_period", ctypes.c_int32), ("store_z", ctypes.c_int32), ("ctas", ctypes.c_int32),
                ("warps_per_cta", ctypes.c_int32), ("min_rows", ctypes.c_int32),
                ("true_residual", ctypes.c_int32), ("maxit_inner", ctypes.c_int32),
                ("max_outer", ctypes.c_int32), ("tol_inner", ctypes.c_double), ("timeout_s", ctypes.c_double),
                ("history", ctypes.c_void_p), ("team_ctas", ctypes.c_int32), ("ring_slots", ctypes.c_int32),
                ("resident", ctypes.c_int32), ("lane_vec", ctypes.c_int32),
                ("reproducible", ctypes.c_int32), ("mg_nu", ctypes.c_int32), ("mg_levels", ctypes.c_int32),
                ("mg_coarse_sweeps", ctypes.c_int32), ("stabilized", ctypes.c_int32)]


_lib = None


def lib():
    """Load liblap5cg.so (building it first when the sources are newer)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH) or os.environ.get("LAP5CG_AUTOBUILD", "1") == "1":
            _build.build()
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("liblap5cg.so is missing; run paper_1803_03797_gb300.build.build()")
        L = ctypes.CDLL(LIB_PATH)
        i, d, vp, sz = ctypes.c_int, ctypes.c_double, ctypes.c_void_p, ctypes.c_size_t
        L.lap5cg_opts_default.argtypes = [ctypes.POINTER(Opts)]
        L.lap5cg_opts_default.restype = None
        L.lap5cg_status_string.argtypes = [i]
        L.lap5cg_status_string.restype = ctypes.c_char_p
        L.lap5_apply.argtypes = [i, i, i, i, vp, vp, vp]
        L.lap5_apply.restype = i
        L.cg_workspace_size.argtypes = [i, i, i, i, i, i]
        L.cg_workspace_size.restype = sz
        L.cg_solve.argtypes = [i, i, i, vp, vp, d, i, i, i, i, vp, sz, vp, ctypes.POINTER(Opts), vp]
        L.cg_solve.restype = i
        IP = ctypes.POINTER(ctypes.c_int)
        VPP = ctypes.POINTER(ctypes.c_void_p)
        L.cg_batched_workspace_size.argtypes = [i, IP, IP, IP, i, i]
        L.cg_batched_workspace_size.restype = sz
        L.cg_solve_batched.argtypes = [i, IP, IP, IP, VPP, VPP, d, i, i, i, vp, sz, vp, ctypes.POINTER(Opts), vp]
        L.cg_solve_batched.restype = i
        L.cg_solve_classic_f64_noalloc.argtypes = [i, i, i, vp, vp, d, i, vp, vp]
        L.cg_solve_classic_f64_noalloc.restype = i
        DP = ctypes.POINTER(ctypes.c_double)
        L.lap5cg_fp64_rate.argtypes = [DP, DP, vp]
        L.lap5cg_fp64_rate.restype = i
        L.lap5cg_release_graphs.argtypes = []
        L.lap5cg_release_graphs.restype = i
        L.lap5cg_tune.argtypes = [i, i, i, vp, vp, i, i, i, vp, sz, vp, ctypes.POINTER(Opts), DP, vp]
        L.lap5cg_tune.restype = i
        L.lap5cg_tune_batched.argtypes = [i, IP, IP, IP, VPP, VPP, i, i, i, vp, sz, vp, ctypes.POINTER(Opts), DP, vp]
        L.lap5cg_tune_batched.restype = i
        _lib = L
    return _lib


EXPORTED = ("lap5cg_opts_default", "lap5cg_status_string", "lap5_apply", "cg_workspace_size", "cg_solve",
            "cg_batched_workspace_size", "cg_solve_batched", "cg_solve_classic_f64_noalloc", "lap5cg_tune",
            "lap5cg_tune_batched", "lap5cg_fp64_rate", "lap5cg_release_graphs")
NOALLOC_MAX_POINTS = 262144


class Lap5cgError(RuntimeError):
    def __init__(self, code, what):
        super().__init__("%s: %s (%d)" % (what, status_string(code), code))
        self.code = code


def status_string(code: int) -> str:
    return lib().lap5cg_status_string(int(code)).decode()


def default_opts(**kw) -> Opts:
    o = Opts()
    lib().lap5cg_opts_default(ctypes.byref(o))
    for k, v in kw.items():
        if not hasattr(o, k):
            raise KeyError(k)
        setattr(o, k, v)
    return o


def _stream(stream, device=None):
    if stream is None:
        stream = torch.cuda.current_stream(device)
    return ctypes.c_void_p(stream.cuda_stream)


def _check_grid(t, name):
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise ValueError("%s must be a CUDA tensor" % name)
    if not t.is_contiguous():
        raise ValueError("%s must be contiguous" % name)


def _check_like(t, ref, name, ref_name="b"):
    """t must be a contiguous CUDA tensor with ref's shape, dtype and device:
    the library reads and writes it with ref's layout."""
    _check_grid(t, name)
    if t.shape != ref.shape or t.dtype != ref.dtype or t.device != ref.device:
        raise ValueError("%s must match %s: shape %s, dtype %s, device %s (got %s, %s, %s)"
                         % (name, ref_name, tuple(ref.shape), ref.dtype, ref.device, tuple(t.shape), t.dtype,
                            t.device))


def _check_info(info, count, device):
    """info must be a contiguous uint8 CUDA tensor of at least count records on device."""
    _check_grid(info, "info")
    if info.dtype != torch.uint8 or info.numel() < count * INFO_BYTES or info.device != device:
        raise ValueError("info must be a uint8 tensor of at least %d bytes on %s" % (count * INFO_BYTES, device))


_DT = {torch.float64: DT_F64, torch.float32: DT_F32, torch.bfloat16: DT_BF16}


def lap5_apply(x: torch.Tensor, nx: int = None, out: torch.Tensor = None, stream=None) -> torch.Tensor:
    """y = A x (Sec. II-B mask, zero Dirichlet boundary) for a (ny, ld) grid."""
    _check_grid(x, "x")
    if x.dim() != 2 or x.dtype not in _DT:
        raise ValueError("x must be a 2D float64/float32/bfloat16 tensor")
    ny, ld = x.shape
    nx = ld if nx is None else int(nx)
    if out is not None:
        _check_like(out, x, "out", "x")
    y = torch.zeros_like(x) if out is None else out
    with torch.cuda.device(x.device):
        rc = lib().lap5_apply(nx, ny, ld, _DT[x.dtype], ctypes.c_void_p(x.data_ptr()),
                              ctypes.c_void_p(y.data_ptr()), _stream(stream, x.device))
    if rc != OK:
        raise Lap5cgError(rc, "lap5_apply")
    return y


def workspace_size(nx, ny, ld, variant="classic", precision="f64", nrhs=1) -> int:
    return int(lib().cg_workspace_size(nx, ny, ld, _VARIANTS[variant], _PRECISIONS[precision], nrhs))


def decode_info(info: torch.Tensor):
    """Device info buffer -> list of dicts (synchronises on the copy)."""
    raw = info.detach().to("cpu").numpy().view(INFO_DTYPE)
    return [{k: (raw[i][k].item()) for k in INFO_DTYPE.names if k != "pad"} for i in range(raw.shape[0])]


def _x_dtype(precision):
    return torch.float32 if _PRECISIONS[precision] == PREC_F32 else torch.float64


def cg_solve(b: torch.Tensor, x0: torch.Tensor = None, tol: float = 1e-10, maxit: int = 10000,
             variant="classic", precision="f64", nx: int = None, opts: Opts = None,
             workspace: torch.Tensor = None, info: torch.Tensor = None, out: torch.Tensor = None,
             stream=None, check: bool = False):
    """Solve A x = b on the GPU (Algorithm 1 or 2) in one persistent launch per
    right-hand side.  b: (ny, ld) or (nrhs, ny, ld).  Returns (x, info) where
    info is a uint8 CUDA tensor of lap5cg_info records (decode_info()).
    check=True synchronises and raises on a non-OK / non-NOT_CONVERGED status."""
    _check_grid(b, "b")
    want = _x_dtype(precision)
    if b.dtype != want:
        raise ValueError("b must be %s for precision %s" % (want, precision))
    if b.dim() == 2:
        nrhs, (ny, ld) = 1, b.shape
    elif b.dim() == 3:
        nrhs, ny, ld = b.shape
    else:
        raise ValueError("b must be (ny, ld) or (nrhs, ny, ld)")
    nx = ld if nx is None else int(nx)
    v, p = _VARIANTS[variant], _PRECISIONS[precision]
    if x0 is not None:
        _check_like(x0, b, "x0")
    if out is not None:
        _check_like(out, b, "out")
        x = out
        if x0 is not None and x0.data_ptr() != x.data_ptr():
            x.copy_(x0)
        elif x0 is None:
            x.zero_()
    else:
        x = torch.zeros_like(b) if x0 is None else x0.clone()
    need = workspace_size(nx, ny, ld, v, p, nrhs)
    if need == 0:
        raise Lap5cgError(ERR_UNSUPPORTED, "cg_workspace_size")
    if workspace is not None:
        _check_grid(workspace, "workspace")
        if workspace.device != b.device:
            raise ValueError("workspace must be on %s" % b.device)
    if workspace is None or workspace.numel() * workspace.element_size() < need:
        workspace = torch.empty(need, dtype=torch.uint8, device=b.device)
    if info is None:
        info = torch.empty(nrhs * INFO_BYTES, dtype=torch.uint8, device=b.device)
    _check_info(info, nrhs, b.device)
    with torch.cuda.device(b.device):
        rc = lib().cg_solve(nx, ny, ld, ctypes.c_void_p(b.data_ptr()), ctypes.c_void_p(x.data_ptr()), float(tol),
                            int(maxit), v, p, nrhs, ctypes.c_void_p(workspace.data_ptr()),
                            workspace.numel() * workspace.element_size(), ctypes.c_void_p(info.data_ptr()),
                            ctypes.byref(opts) if opts is not None else None, _stream(stream, b.device))
    if rc != OK:
        raise Lap5cgError(rc, "cg_solve")
    if check:
        for rec in decode_info(info):
            if rec["status"] < 0:
                raise Lap5cgError(rec["status"], "cg_solve (device)")
    return x, info


def batched_workspace_size(nx_list, ny_list, ld_list, variant="classic", precision="ir_f32") -> int:
    n = len(nx_list)
    arr = ctypes.c_int * n
    return int(lib().cg_batched_workspace_size(n, arr(*nx_list), arr(*ny_list), arr(*ld_list), _VARIANTS[variant],
                                               _PRECISIONS[precision]))


def cg_solve_batched(bs, xs=None, tol=1e-10, maxit=100000, variant="classic", precision="ir_f32", nx_list=None,
                     opts: Opts = None, workspace=None, info=None, stream=None):
    """Solve len(bs) independent systems of different shapes in one persistent
    launch.  bs: list of (ny, ld) CUDA tensors.  Returns (xs, info)."""
    n = len(bs)
    if n < 1:
        raise ValueError("empty batch")
    dev = bs[0].device
    for t in bs:
        _check_grid(t, "b")
        if t.dim() != 2 or t.device != dev:
            raise ValueError("every b must be a 2D tensor on %s" % dev)
    nxs = [t.shape[1] for t in bs] if nx_list is None else list(nx_list)
    nys = [t.shape[0] for t in bs]
    lds = [t.shape[1] for t in bs]
    if xs is None:
        xs = [torch.zeros_like(t) for t in bs]
    if len(xs) != n:
        raise ValueError("xs must have one tensor per b")
    for t, bt in zip(xs, bs):
        _check_like(t, bt, "x")
    v, p = _VARIANTS[variant], _PRECISIONS[precision]
    need = batched_workspace_size(nxs, nys, lds, v, p)
    if need == 0:
        raise Lap5cgError(ERR_UNSUPPORTED, "cg_batched_workspace_size")
    if workspace is not None:
        _check_grid(workspace, "workspace")
        if workspace.device != dev:
            raise ValueError("workspace must be on %s" % dev)
    if workspace is None or workspace.numel() * workspace.element_size() < need:
        workspace = torch.empty(need, dtype=torch.uint8, device=dev)
    if info is None:
        info = torch.empty(n * INFO_BYTES, dtype=torch.uint8, device=dev)
    _check_info(info, n, dev)
    arr = ctypes.c_int * n
    ptrs = ctypes.c_void_p * n
    with torch.cuda.device(dev):
        rc = lib().cg_solve_batched(n, arr(*nxs), arr(*nys), arr(*lds), ptrs(*[t.data_ptr() for t in bs]),
                                    ptrs(*[t.data_ptr() for t in xs]), float(tol), int(maxit), v, p,
                                    ctypes.c_void_p(workspace.data_ptr()), workspace.numel() * workspace.element_size(),
                                    ctypes.c_void_p(info.data_ptr()),
                                    ctypes.byref(opts) if opts is not None else None, _stream(stream, dev))
    if rc != OK:
        raise Lap5cgError(rc, "cg_solve_batched")
    return xs, info


def cg_solve_classic_f64_noalloc(b: torch.Tensor, x0: torch.Tensor = None, tol: float = 1e-10, maxit: int = 10000,
                                 nx: int = None, out: torch.Tensor = None, info: torch.Tensor = None, stream=None):
    """Classic binary64 CG through the entry point that allocates no device
    memory (scratch lives in a fixed array inside the library; ny*ld must not
    exceed NOALLOC_MAX_POINTS).  Returns (x, info)."""
    _check_grid(b, "b")
    if b.dtype != torch.float64 or b.dim() != 2:
        raise ValueError("b must be a 2D float64 CUDA tensor")
    ny, ld = b.shape
    nx = ld if nx is None else int(nx)
    if x0 is not None:
        _check_like(x0, b, "x0")
    if out is not None:
        _check_like(out, b, "out")
    x = out if out is not None else torch.zeros_like(b)
    if x0 is not None:
        if x0.data_ptr() != x.data_ptr():
            x.copy_(x0)
    elif out is not None:
        x.zero_()
    if info is None:
        info = torch.empty(INFO_BYTES, dtype=torch.uint8, device=b.device)
    _check_info(info, 1, b.device)
    with torch.cuda.device(b.device):  # the library's scratch array is looked up on the current device
        rc = lib().cg_solve_classic_f64_noalloc(nx, ny, ld, ctypes.c_void_p(b.data_ptr()),
                                                ctypes.c_void_p(x.data_ptr()), float(tol), int(maxit),
                                                ctypes.c_void_p(info.data_ptr()), _stream(stream, b.device))
    if rc != OK:
        raise Lap5cgError(rc, "cg_solve_classic_f64_noalloc")
    return x, info


def release_graphs():
    """Free the library's cached multigrid graphs on every device (before a
    device reset; the next classic multigrid solve builds its graph again)."""
    rc = lib().lap5cg_release_graphs()
    if rc != OK:
        raise Lap5cgError(rc, "lap5cg_release_graphs")


def fp64_rate(device=None):
    """Measured binary64 lane-operation rates of the GPU: {"fma_per_s", "add_per_s"}
    (a throughput kernel timed on the device; synchronises)."""
    dev = torch.device("cuda", torch.cuda.current_device()) if device is None else torch.device(device)
    f, a = ctypes.c_double(), ctypes.c_double()
    with torch.cuda.device(dev):
        rc = lib().lap5cg_fp64_rate(ctypes.byref(f), ctypes.byref(a), _stream(None, dev))
    if rc != OK:
        raise Lap5cgError(rc, "lap5cg_fp64_rate")
    return {"fma_per_s": f.value, "add_per_s": a.value}


# ---------------------------------------------------------------------------
# Autotuning: lap5cg_tune picks launch parameters by timing real solves; the
# results are cached in a JSON file keyed by GPU name, precision, variant and
# a size class (powers of two of the grid sides).
# ---------------------------------------------------------------------------
_OPT_FIELDS = ("warps_per_cta", "ring_slots", "min_rows", "store_z", "team_ctas", "ctas", "resident", "lane_vec")


def _cache_path():
    return os.environ.get("LAP5CG_TUNE_CACHE",
                          os.path.join(os.path.expanduser("~"), ".cache", "lap5cg", "tune.json"))


def size_class(nx, ny):
    return "%dx%d" % (1 << max(0, int(nx - 1).bit_length()), 1 << max(0, int(ny - 1).bit_length()))


def _key(kind, variant, precision, nx, ny):
    dev = torch.cuda.get_device_name()
    return "|".join([dev, kind, str(variant), str(precision), size_class(nx, ny)])


def _load_cache():
    import json
    try:
        with open(_cache_path()) as f:
            return json.load(f)
    except Exception:
        return {}


def _store_cache(key, opts, ms):
    import json
    d = _load_cache()
    d[key] = {"opts": {k: int(getattr(opts, k)) for k in _OPT_FIELDS}, "ms": ms}
    path = _cache_path()
    os.makedirs(os.path.dirname(path), exist_ok=True)
    tmp = path + ".tmp%d" % os.getpid()
    with open(tmp, "w") as f:
        json.dump(d, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def tuned_opts(nx, ny, variant="classic", precision="f64", batched=False):
    """Options from the tuning cache for this size class, or None."""
    rec = _load_cache().get(_key("batched" if batched else "single", variant, precision, nx, ny))
    if not rec:
        return None
    return default_opts(**rec["opts"])


def autotune(b: torch.Tensor, variant="classic", precision="f64", iters=100, nx=None, start: Opts = None,
             cache=True, stream=None):
    """Tune launch parameters for solves shaped like b; returns (opts, ms)."""
    _check_grid(b, "b")
    ny, ld = b.shape
    nx = ld if nx is None else int(nx)
    v, p = _VARIANTS[variant], _PRECISIONS[precision]
    x = torch.zeros_like(b)
    ws = torch.empty(workspace_size(nx, ny, ld, v, p), dtype=torch.uint8, device=b.device)
    info = torch.empty(INFO_BYTES, dtype=torch.uint8, device=b.device)
    o = start if start is not None else default_opts()
    ms = ctypes.c_double()
    with torch.cuda.device(b.device):
        rc = lib().lap5cg_tune(nx, ny, ld, ctypes.c_void_p(b.data_ptr()), ctypes.c_void_p(x.data_ptr()), v, p,
                               int(iters), ctypes.c_void_p(ws.data_ptr()), ws.numel(),
                               ctypes.c_void_p(info.data_ptr()), ctypes.byref(o), ctypes.byref(ms),
                               _stream(stream, b.device))
    if rc != OK:
        raise Lap5cgError(rc, "lap5cg_tune")
    if cache:
        _store_cache(_key("single", variant, precision, nx, ny), o, ms.value)
    return o, ms.value


def autotune_batched(bs, variant="classic", precision="ir_f32", iters=100, nx_list=None, start: Opts = None,
                     cache=True, stream=None):
    """Tune team size and launch parameters for a batch shaped like bs."""
    n = len(bs)
    nxs = [t.shape[1] for t in bs] if nx_list is None else list(nx_list)
    nys = [t.shape[0] for t in bs]
    lds = [t.shape[1] for t in bs]
    v, p = _VARIANTS[variant], _PRECISIONS[precision]
    xs = [torch.zeros_like(t) for t in bs]
    ws = torch.empty(batched_workspace_size(nxs, nys, lds, v, p), dtype=torch.uint8, device=bs[0].device)
    info = torch.empty(n * INFO_BYTES, dtype=torch.uint8, device=bs[0].device)
    o = start if start is not None else default_opts()
    ms = ctypes.c_double()
    arr = ctypes.c_int * n
    ptrs = ctypes.c_void_p * n
    with torch.cuda.device(bs[0].device):
        rc = lib().lap5cg_tune_batched(n, arr(*nxs), arr(*nys), arr(*lds), ptrs(*[t.data_ptr() for t in bs]),
                                       ptrs(*[t.data_ptr() for t in xs]), v, p, int(iters),
                                       ctypes.c_void_p(ws.data_ptr()), ws.numel(), ctypes.c_void_p(info.data_ptr()),
                                       ctypes.byref(o), ctypes.byref(ms), _stream(stream, bs[0].device))
    if rc != OK:
        raise Lap5cgError(rc, "lap5cg_tune_batched")
    if cache:
        _store_cache(_key("batched", variant, precision, max(nxs), max(nys)), o, ms.value)
    return o, ms.value


class CGSolve(torch.autograd.Function):
    """x = A^{-1} b by CG on the GPU; backward is the adjoint solve
    grad_b = A^{-1} grad_x (A is symmetric), a second CG solve with the same
    settings.  Nothing but the settings is saved for backward."""

    @staticmethod
    def forward(ctx, b, tol=1e-10, maxit=100000, variant="classic", precision="f64", nx=None):
        ctx.settings = (tol, maxit, variant, precision, nx)
        x, info = cg_solve(b.detach(), tol=tol, maxit=maxit, variant=variant, precision=precision, nx=nx)
        ctx.mark_non_differentiable(info)
        return x, info

    @staticmethod
    def backward(ctx, grad_x, grad_info):
        tol, maxit, variant, precision, nx = ctx.settings
        g, _ = cg_solve(grad_x.contiguous(), tol=tol, maxit=maxit, variant=variant, precision=precision, nx=nx)
        return g, None, None, None, None, None


def solve(b, tol=1e-10, maxit=100000, variant="classic", precision="f64", nx=None):
    """Differentiable solve: returns x only."""
    x, _ = CGSolve.apply(b, tol, maxit, variant, precision, nx)
    return x
