"""Pins for the oracle's reproducible mode: the reproducible dot product and
Algorithms 1 / 2 built on it.

The dot product is defined by four steps (blocks of 2 columns x 16 rows; row
value fma(a1, b1, a0*b0); a fixed pairwise tree per block; the exact sum of
the block values rounded once).  The references here are independent of the
oracle's code: a pure-Python restatement with exact rational arithmetic
(fractions.Fraction) for the fused multiply-add and for the exact sum, exact
integer dot products, the rounding-error bound of the definition, and the
textbook solves already used for the default mode (dense Cholesky, the
closed-form one-step case).
"""
import math
from fractions import Fraction

import numpy as np
import pytest
import scipy.linalg as sla

import lap5_inputs as gen
import oracle
from tests.helpers import flat, kron_laplacian

U = 2.0 ** -53


def _fma(a, b, c):
    return float(Fraction(a) * Fraction(b) + Fraction(c))


def _blocks_py(a, b, nx, ny):
    """Steps 1-3 restated in Python with exact rational fused multiply-adds."""
    nbx, nby = (nx + 1) // 2, (ny + 15) // 16
    out = np.zeros((nby, nbx))
    for t in range(nby):
        for c in range(nbx):
            v = []
            for m in range(16):
                j = 16 * t + m
                if j >= ny:
                    v.append(0.0)
                    continue
                a0, b0 = float(a[j, 2 * c]), float(b[j, 2 * c])
                a1 = float(a[j, 2 * c + 1]) if 2 * c + 1 < nx else 0.0
                b1 = float(b[j, 2 * c + 1]) if 2 * c + 1 < nx else 0.0
                v.append(_fma(a1, b1, a0 * b0))
            while len(v) > 1:
                v = [v[2 * m] + v[2 * m + 1] for m in range(len(v) // 2)]
            out[t, c] = v[0]
    return out


def _grid_pair(nx, ny, seed, pad=3):
    rng = np.random.default_rng(seed)
    ld = nx + pad
    a = rng.standard_normal((ny, ld)) * np.exp(rng.uniform(-20, 20, (ny, ld)))
    b = rng.standard_normal((ny, ld))
    a[:, nx:] = 1e300  # padding columns are not part of the grid
    b[:, nx:] = -7.0
    return a, b


SHAPES = [(1, 1), (2, 1), (3, 5), (7, 16), (33, 17), (20, 40), (5, 15)]


@pytest.mark.parametrize("nx,ny", SHAPES)
def test_blocks_match_rational_restatement(nx, ny):
    a, b = _grid_pair(nx, ny, seed=nx * 7 + ny)
    got = oracle.repro_blocks(a, b, nx=nx)
    ref = _blocks_py(a, b, nx, ny)
    assert got.shape == ref.shape
    assert np.array_equal(got, ref)


@pytest.mark.parametrize("nx,ny", SHAPES)
def test_dot_is_correctly_rounded_exact_block_sum(nx, ny):
    a, b = _grid_pair(nx, ny, seed=nx * 11 + ny)
    ref = float(sum((Fraction(float(v)) for v in _blocks_py(a, b, nx, ny).ravel()), Fraction(0)))
    assert oracle.dot_repro(a, b, nx=nx) == ref


def test_exact_sum_cancellation_and_range():
    # values spanning the binary64 range with heavy cancellation
    rng = np.random.default_rng(3)
    vals = list(rng.standard_normal(200) * np.exp2(rng.integers(-1000, 1000, 200)))
    vals += [-v for v in vals[:150]] + [2.0 ** -1074, 3 * 2.0 ** -1074, 1e308, -1e308, 0.5, 2.0 ** -60]
    exact = sum((Fraction(v) for v in vals), Fraction(0))
    assert oracle.exact_sum(vals) == float(exact)
    # ties round to even: 1 + 2^-53 is halfway between 1 and 1 + 2^-52
    assert oracle.exact_sum([1.0, 2.0 ** -53]) == 1.0
    assert oracle.exact_sum([1.0, 2.0 ** -53, 2.0 ** -200]) == 1.0 + 2.0 ** -52
    assert oracle.exact_sum([1.0 + 2.0 ** -52, 2.0 ** -53]) == 1.0 + 2.0 ** -51


def test_dot_special_values():
    z = np.zeros((20, 6))
    assert math.copysign(1.0, oracle.dot_repro(z, -z)) == 1.0  # exact zero is +0
    a = np.ones((20, 6))
    b = -np.ones((20, 6))
    b[3, 2] = 0.0
    assert oracle.dot_repro(a, b) == -119.0
    a[7, 5] = np.inf
    assert math.isnan(oracle.dot_repro(a, np.ones((20, 6))))
    a[7, 5] = np.nan
    assert math.isnan(oracle.dot_repro(a, np.ones((20, 6))))


@pytest.mark.parametrize("nx,ny", [(31, 33), (64, 64), (100, 17)])
def test_integer_inputs_give_the_exact_integer_dot(nx, ny):
    rng = np.random.default_rng(nx + ny)
    a = rng.integers(-1000, 1000, (ny, nx)).astype(np.float64)
    b = rng.integers(-1000, 1000, (ny, nx)).astype(np.float64)
    exact = int(np.sum(a.astype(np.int64) * b.astype(np.int64)))
    assert oracle.dot_repro(a, b) == float(exact)


@pytest.mark.parametrize("nx,ny", [(50, 50), (129, 40)])
def test_dot_error_within_the_definitions_bound(nx, ny):
    rng = np.random.default_rng(nx)
    a = rng.standard_normal((ny, nx))
    b = rng.standard_normal((ny, nx))
    exact = sum((Fraction(float(x)) * Fraction(float(y)) for x, y in zip(a.ravel(), b.ravel())), Fraction(0))
    got = oracle.dot_repro(a, b)
    # per term: one rounding of a0*b0, one of the fma, four tree levels; then one final rounding
    bound = 7 * U * float(np.sum(np.abs(a * b))) * 1.01 + U * abs(float(exact))
    assert abs(Fraction(got) - exact) <= Fraction(bound)


def test_dot_differs_from_sequential_order_only_by_rounding():
    b = gen.uniform_rhs(300, 200, seed=9)
    d1, d2 = oracle.dot_repro(b, b), oracle.dot(b, b)
    assert abs(d1 - d2) <= 1e-12 * d2


@pytest.mark.parametrize("variant", ["classic", "newcg"])
@pytest.mark.parametrize("nx,ny", [(2, 2), (3, 5), (16, 16), (16, 7)])
def test_repro_cg_dense_cholesky(variant, nx, ny):
    A = kron_laplacian(nx, ny).toarray()
    b = gen.uniform_rhs(nx, ny, seed=nx * 100 + ny)
    x_ref = sla.cho_solve(sla.cho_factor(A), flat(b, nx))
    fn = oracle.cg_classic_repro if variant == "classic" else oracle.cg_newcg_repro
    x, info = fn(b, tol=1e-13, maxit=10 * nx * ny)
    assert info["status"] == oracle.OK
    err = np.linalg.norm(flat(x, nx) - x_ref) / np.linalg.norm(x_ref)
    assert err <= gen.condition_number(nx, ny) * 1e-13 * 4


@pytest.mark.parametrize("variant", ["classic", "newcg"])
def test_repro_cg_single_eigenvector_terminates_in_one_step(variant):
    n = 40
    lam = gen.mode_eigenvalue(n, n, 1, 1)
    u = gen.sine_mode(n, n, 1, 1)
    fn = oracle.cg_classic_repro if variant == "classic" else oracle.cg_newcg_repro
    x, info = fn(lam * u, tol=1e-12, maxit=10)
    assert info["iters"] == 1 and info["status"] == oracle.OK
    assert np.abs(x - u).max() <= 1e-13


@pytest.mark.parametrize("variant", ["classic", "newcg"])
@pytest.mark.parametrize("nx,ny,k", [(100, 100, 30), (33, 70, 25), (1, 40, 10)])
def test_repro_cg_tracks_default_mode(variant, nx, ny, k):
    # the two modes differ only in rounding (dot order, fused updates)
    b = gen.uniform_rhs(nx, ny, seed=nx + 3 * ny)
    fn = oracle.cg_classic_repro if variant == "classic" else oracle.cg_newcg_repro
    x, info = fn(b, tol=0.0, maxit=k)
    xo, io = oracle.cg_solve(b, variant=variant, tol=0.0, maxit=k)
    assert info["iters"] == io["iters"]
    assert np.linalg.norm(x - xo) <= 1e-11 * np.linalg.norm(xo)


def test_repro_newcg_matches_repro_classic_early():
    b = gen.uniform_rhs(64, 64, seed=4)
    for k in (1, 5, 20):
        xc, _ = oracle.cg_classic_repro(b, tol=0.0, maxit=k)
        xn, _ = oracle.cg_newcg_repro(b, tol=0.0, maxit=k)
        assert np.linalg.norm(xc - xn) <= 1e-10 * np.linalg.norm(xc)


def test_repro_newcg_residual_replacement_keeps_the_iterate():
    b = gen.uniform_rhs(48, 48, seed=6)
    x0, _ = oracle.cg_newcg_repro(b, tol=0.0, maxit=40)
    x1, _ = oracle.cg_newcg_repro(b, tol=0.0, maxit=40, rr_period=10)
    assert np.linalg.norm(x0 - x1) <= 1e-9 * np.linalg.norm(x0)


def test_repro_first_step_by_hand():
    # x1 = alpha r0 with alpha = (r0, r0) / (r0, A r0), both dots by definition
    b = gen.uniform_rhs(9, 20, seed=12)
    x, info = oracle.cg_classic_repro(b, tol=0.0, maxit=1)
    ab = oracle.lap5_apply(b)
    gamma = float(sum((Fraction(float(v)) for v in _blocks_py(b, b, 9, 20).ravel()), Fraction(0)))
    pz = float(sum((Fraction(float(v)) for v in _blocks_py(b, ab, 9, 20).ravel()), Fraction(0)))
    alpha = gamma / pz
    assert np.array_equal(x, alpha * b)  # fma(alpha, p, 0) = alpha * p rounded once
