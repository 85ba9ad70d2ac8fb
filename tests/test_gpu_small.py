"""Cluster-resident solves (the whole grid in one thread-block cluster's shared
memory) at the paper's grid sizes (Sec. III: N = 16, 32, 40, 100) and other
small shapes, against the oracle and against the streaming kernels."""
import numpy as np
import pytest
import torch

import lap5_inputs as gen
import oracle
import paper_1803_03797_gb300 as lap5cg
from tests.helpers import rel_err

pytestmark = pytest.mark.gpu

VARIANTS = ["classic", "newcg"]
SHAPES = [(16, 16), (32, 32), (40, 40), (100, 100), (1, 1), (1, 7), (7, 1), (3, 5), (17, 300), (250, 250), (255, 31)]


def _rel(a, b):
    return rel_err(a, b)  # norm-wise and element-wise


def _solve(b, nx, **kw):
    x, info = lap5cg.cg_solve(torch.from_numpy(b).cuda(), nx=nx, **kw)
    return x.cpu().numpy(), lap5cg.decode_info(info)[0]


@pytest.mark.parametrize("variant", VARIANTS)
@pytest.mark.parametrize("nx,ny", SHAPES)
def test_resident_f64_matches_oracle(variant, nx, ny):
    b = gen.uniform_rhs(nx, ny, seed=3 * nx + ny, ld=gen.pitch(nx, 8))
    k = min(30, nx * ny - 1) if nx * ny > 1 else 1
    x, rec = _solve(b, nx, tol=0.0, maxit=k, variant=variant)
    xo, io = oracle.cg_solve(b, variant=variant, tol=0.0, maxit=k, nx=nx)
    assert rec["iters"] == io["iters"]
    assert _rel(x[:, :nx], xo[:, :nx]) <= 1e-10
    x, rec = _solve(b, nx, tol=1e-10, maxit=20000, variant=variant)
    xo, io = oracle.cg_solve(b, variant=variant, tol=1e-10, maxit=20000, nx=nx)
    assert rec["status"] == lap5cg.OK and abs(rec["iters"] - io["iters"]) <= 2
    assert rec["relres_true"] <= 3 * max(io["relres_true"], 1e-10)


@pytest.mark.parametrize("variant", VARIANTS)
@pytest.mark.parametrize("nx,ny", [(100, 100), (40, 40), (129, 60)])
def test_resident_equals_streaming(variant, nx, ny):
    b = gen.uniform_rhs(nx, ny, seed=nx + ny, ld=gen.pitch(nx, 8))
    xa, ra = _solve(b, nx, tol=0.0, maxit=50, variant=variant)
    xb, rb = _solve(b, nx, tol=0.0, maxit=50, variant=variant, opts=lap5cg.default_opts(resident=-1))
    assert _rel(xa[:, :nx], xb[:, :nx]) <= 1e-10  # dot sums differ in order only


@pytest.mark.parametrize("variant", VARIANTS)
def test_resident_f32(variant):
    n = 100
    b = gen.uniform_rhs(n, n, seed=9).astype(np.float32)
    x, rec = _solve(b, n, tol=0.0, maxit=30, variant=variant, precision="f32")
    xo, io = oracle.cg_solve(b.astype(np.float64), variant=variant, tol=0.0, maxit=30)
    assert _rel(x.astype(np.float64), xo) <= (1e-4 if variant == "classic" else 1e-3)


@pytest.mark.parametrize("variant", VARIANTS)
def test_resident_edge_cases(variant):
    n = 32
    z = np.zeros((n, n))
    x, rec = _solve(z, n, x0=torch.ones(n, n, dtype=torch.float64).cuda(), tol=1e-8, maxit=10, variant=variant)
    assert rec["status"] == lap5cg.OK and rec["iters"] == 0 and not x.any()
    b = gen.uniform_rhs(n, n, seed=1)
    b[3, 3] = np.nan
    x, rec = _solve(b, n, tol=1e-8, maxit=10, variant=variant)
    assert rec["status"] == lap5cg.ERR_NONFINITE
    lam = gen.mode_eigenvalue(n, n, 1, 1)
    u = gen.sine_mode(n, n, 1, 1)
    x, rec = _solve(lam * u, n, tol=1e-12, maxit=5, variant=variant)
    assert rec["iters"] == 1 and np.abs(x - u).max() <= 1e-13
