"""Seeded synthetic inputs for the 2D Dirichlet 5-point Laplacian CG workloads.

This module is shared by the CPU oracle's tests and by the GPU path's tests and
benchmark.  It holds input construction only (random draws, grid coordinates,
closed-form modes) and none of the solver's arithmetic: no stencil, no dot
product, no CG step.

Conventions: a grid is an array of shape (ny, ld) with ld >= nx (row pitch in
elements); element (i, j) is ``a[j, i]``; padding columns i >= nx are zero.
Interior point (i, j) (0-based) sits at x = (i+1)/(nx+1), y = (j+1)/(ny+1)
(Sec. II: points 1 <= i, j <= n of the unit square).

Random numbers come from ``numpy.random.default_rng(seed)`` (PCG64).
"""
import math

import numpy as np

# Workloads the paper measures (Sec. III: N x N grids with N in {16, 32, 40,
# 100}) extended to GPU scale; each entry is (name, description, seed).
WORKLOADS = {
    "c1_100": dict(nx=100, ny=100, seed=1, rhs="uniform", dtype="f64", tol=1e-8),
    "c2_4096": dict(nx=4096, ny=4096, seed=2, rhs="manufactured", dtype="f64", fixed_iters=500, tol=1e-10),
    "c3_8192": dict(nx=8192, ny=8192, seed=3, rhs="uniform", dtype="f64", tol=1e-10),
    "c4_batched": dict(count=256, lo=64, hi=1024, seed=4, rhs="uniform"),
    "c5_grad": dict(nx=2048, ny=2048, nrhs=16, seed=5),
}


def pitch(nx: int, elem_bytes: int, align_bytes: int = 16) -> int:
    """Smallest ld >= nx whose row size is a multiple of align_bytes."""
    per = max(1, align_bytes // elem_bytes)
    return ((nx + per - 1) // per) * per


def _place(core: np.ndarray, ld: int) -> np.ndarray:
    ny, nx = core.shape
    out = np.zeros((ny, ld), dtype=core.dtype)
    out[:, :nx] = core
    return out


def uniform_rhs(nx: int, ny: int, seed: int, ld: int = None, dtype=np.float64) -> np.ndarray:
    """b_ij ~ U[-1, 1) i.i.d., drawn row by row as 2*random() - 1."""
    rng = np.random.default_rng(seed)
    core = 2.0 * rng.random((ny, nx)) - 1.0
    return _place(core.astype(dtype), ld if ld is not None else nx)


def gaussian_field(nx: int, ny: int, seed: int, ld: int = None, dtype=np.float64) -> np.ndarray:
    """i.i.d. standard normal values (e.g. a target x for the gradient workload)."""
    rng = np.random.default_rng(seed)
    core = rng.standard_normal((ny, nx))
    return _place(core.astype(dtype), ld if ld is not None else nx)


def coords(nx: int, ny: int):
    """Interior grid coordinates x_i = (i+1)/(nx+1), y_j = (j+1)/(ny+1)."""
    xs = np.arange(1, nx + 1, dtype=np.float64) / (nx + 1)
    ys = np.arange(1, ny + 1, dtype=np.float64) / (ny + 1)
    return xs, ys


def sine_mode(nx: int, ny: int, k: int = 1, l: int = 1, ld: int = None) -> np.ndarray:
    """v_ij = sin(k*pi*x_i) * sin(l*pi*y_j), 1 <= k <= nx, 1 <= l <= ny."""
    xs, ys = coords(nx, ny)
    core = np.outer(np.sin(l * math.pi * ys), np.sin(k * math.pi * xs))
    return _place(core, ld if ld is not None else nx)


def mode_eigenvalue(nx: int, ny: int, k: int = 1, l: int = 1) -> float:
    """Closed-form eigenvalue 4 - 2cos(k pi/(nx+1)) - 2cos(l pi/(ny+1)) of the
    unscaled 5-point Dirichlet Laplacian for the sine mode (k, l)."""
    return 4.0 - 2.0 * math.cos(k * math.pi / (nx + 1)) - 2.0 * math.cos(l * math.pi / (ny + 1))


def condition_number(nx: int, ny: int) -> float:
    lo = mode_eigenvalue(nx, ny, 1, 1)
    hi = mode_eigenvalue(nx, ny, nx, ny)
    return hi / lo


def manufactured_rhs(nx: int, ny: int, seed: int, noise: float = 1e-3, ld: int = None) -> np.ndarray:
    """b = A u* + noise * xi with u* = sin(pi x) sin(pi y) and xi ~ N(0, 1).

    u* is the (1, 1) sine mode, so A u* equals lambda_11 u* in exact arithmetic;
    b is formed as lambda_11 * u* + noise * xi (no stencil is applied here)."""
    u = sine_mode(nx, ny, 1, 1)
    lam = mode_eigenvalue(nx, ny, 1, 1)
    rng = np.random.default_rng(seed)
    xi = rng.standard_normal((ny, nx))
    return _place(lam * u + noise * xi, ld if ld is not None else nx)


def batched_shapes(count: int = 256, lo: int = 64, hi: int = 1024, seed: int = 4):
    """Side lengths nx, ny drawn independently and uniformly from {lo..hi}."""
    rng = np.random.default_rng(seed)
    nx = rng.integers(lo, hi + 1, size=count)
    ny = rng.integers(lo, hi + 1, size=count)
    return [int(v) for v in nx], [int(v) for v in ny]


def batched_rhs(nx_list, ny_list, seed: int = 4, elem_bytes: int = 8, dtype=np.float64, align_bytes: int = 32):
    """One U[-1,1) right-hand side per instance, seeded seed*1000003 + k, rows
    padded to a multiple of align_bytes."""
    out = []
    for k, (nx, ny) in enumerate(zip(nx_list, ny_list)):
        out.append(uniform_rhs(nx, ny, seed * 1000003 + k, ld=pitch(nx, elem_bytes, align_bytes), dtype=dtype))
    return out
