"""GPU reproducible mode (opts.reproducible = 1) against the oracle's
reproducible Algorithms 1 and 2: bit-identical iterates.

In this mode every dot product is the exact sum of fixed 2 x 16 block values
rounded once, and every vector update is a single-rounding fused multiply-add,
in the oracle and on the GPU alike; the stencil is already bit-exact.  So the
whole CG trajectory -- x, the residual norms, the iteration count -- must agree
bit for bit with the oracle, and must not change with the launch configuration
(CTAs, warps per CTA, ring slots, unit heights)."""
import numpy as np
import pytest
import torch

import lap5_inputs as gen
import oracle
import paper_1803_03797_gb300 as lap5cg

pytestmark = pytest.mark.gpu


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda")


def _solve(b, nx, variant, tol, maxit, **opt):
    opts = lap5cg.default_opts(reproducible=1, **opt)
    x, info = lap5cg.cg_solve(_dev(b), tol=tol, maxit=maxit, variant=variant, nx=nx, opts=opts)
    return x.cpu().numpy()[:, :nx], lap5cg.decode_info(info)[0]


def _oracle(b, nx, variant, tol, maxit, rr_period=0):
    if variant == "classic":
        x, io = oracle.cg_classic_repro(b, tol=tol, maxit=maxit, nx=nx)
    else:
        x, io = oracle.cg_newcg_repro(b, tol=tol, maxit=maxit, nx=nx, rr_period=rr_period)
    return x[:, :nx], io


def _same(rec, io):
    assert rec["iters"] == io["iters"], (rec, io)
    assert rec["status"] == io["status"], (rec, io)
    assert rec["relres_recursive"] == io["relres_recursive"], (rec, io)
    assert rec["relres_true"] == io["relres_true"], (rec, io)


SHAPES = [(1, 1), (2, 3), (3, 5), (16, 16), (17, 33), (64, 15), (100, 100), (130, 67), (255, 257), (301, 170)]


@pytest.mark.parametrize("variant", ["classic", "newcg"])
@pytest.mark.parametrize("nx,ny", SHAPES)
def test_fixed_iterations_bit_identical_to_oracle(variant, nx, ny):
    b = gen.uniform_rhs(nx, ny, seed=nx * 13 + ny, ld=gen.pitch(nx, 8))
    k = 25
    x, rec = _solve(b, nx, variant, 0.0, k)
    xo, io = _oracle(b, nx, variant, 0.0, k)
    _same(rec, io)
    assert np.array_equal(x, xo)


@pytest.mark.parametrize("variant", ["classic", "newcg"])
@pytest.mark.parametrize("nx,ny", [(100, 100), (130, 67)])
def test_converged_solve_bit_identical_to_oracle(variant, nx, ny):
    b = gen.uniform_rhs(nx, ny, seed=nx + 7 * ny, ld=gen.pitch(nx, 8))
    x, rec = _solve(b, nx, variant, 1e-10, 20000)
    xo, io = _oracle(b, nx, variant, 1e-10, 20000)
    assert rec["status"] == lap5cg.OK
    _same(rec, io)
    assert np.array_equal(x, xo)


def test_newcg_residual_replacement_bit_identical_to_oracle():
    nx, ny = 150, 90
    b = gen.uniform_rhs(nx, ny, seed=31, ld=gen.pitch(nx, 8))
    x, rec = _solve(b, nx, "newcg", 0.0, 60, rr_period=20)
    xo, io = _oracle(b, nx, "newcg", 0.0, 60, rr_period=20)
    _same(rec, io)
    assert np.array_equal(x, xo)


LAUNCHES = [dict(), dict(ctas=37), dict(ctas=152, warps_per_cta=8), dict(warps_per_cta=16, ring_slots=3),
            dict(ring_slots=-1), dict(ring_slots=8, min_rows=40), dict(ctas=5, warps_per_cta=1)]


@pytest.mark.parametrize("variant", ["classic", "newcg"])
def test_launch_configuration_does_not_change_the_result(variant):
    nx, ny = 700, 509
    b = gen.uniform_rhs(nx, ny, seed=44, ld=gen.pitch(nx, 8))
    ref = None
    for opt in LAUNCHES:
        x, rec = _solve(b, nx, variant, 0.0, 40, **opt)
        if ref is None:
            ref = (x, rec)
            xo, io = _oracle(b, nx, variant, 0.0, 40)
            _same(rec, io)
            assert np.array_equal(x, xo)
        else:
            assert np.array_equal(x, ref[0]), opt
            assert rec == ref[1], opt
    if variant == "classic":  # z stored or A p recomputed: the same operands
        x, rec = _solve(b, nx, variant, 0.0, 40, store_z=0)
        assert np.array_equal(x, ref[0]) and rec == ref[1]


@pytest.mark.parametrize("variant", ["classic", "newcg"])
def test_full_size_4096_bit_identical_to_oracle(variant):
    # the benchmark's 4096 x 4096 grid and right-hand side in its launch
    # configuration, reproducible mode, 12 iterations
    n, k = 4096, 12
    b = gen.manufactured_rhs(n, n, seed=2)
    x, rec = _solve(b, n, variant, 0.0, k)
    xo, io = _oracle(b, n, variant, 0.0, k)
    _same(rec, io)
    assert np.array_equal(x, xo)


def test_reproducible_edge_cases_and_rejections():
    n = 40
    z = np.zeros((n, n))
    x, rec = _solve(z, n, "classic", 1e-10, 100)
    assert rec["status"] == lap5cg.OK and rec["iters"] == 0 and not x.any()
    b = gen.uniform_rhs(n, n, seed=1)
    b[3, 4] = np.nan
    x, rec = _solve(b, n, "newcg", 1e-10, 100)
    assert rec["status"] == lap5cg.ERR_NONFINITE
    b = _dev(gen.uniform_rhs(n, n, seed=1))
    with pytest.raises(lap5cg.Lap5cgError):  # binary32: unsupported
        lap5cg.cg_solve(b.float(), tol=1e-5, precision="f32", opts=lap5cg.default_opts(reproducible=1))
    with pytest.raises(lap5cg.Lap5cgError):  # not a flag value
        lap5cg.cg_solve(b, tol=1e-5, opts=lap5cg.default_opts(reproducible=2))
    with pytest.raises(lap5cg.Lap5cgError):  # batched: unsupported
        lap5cg.cg_solve_batched([b, b], tol=1e-8, precision="f64", opts=lap5cg.default_opts(reproducible=1))
