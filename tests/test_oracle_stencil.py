"""Pins for the oracle's stencil (Sec. II-B mask, zero Dirichlet boundary).

Each test checks the oracle against something other than itself: the mask the
paper prints, an independently assembled sparse matrix (Kronecker sum), the
closed-form eigenpairs, and a library bf16 conversion.
"""
import math
import os

import numpy as np
import pytest
import torch

import lap5_inputs as gen
import oracle
from tests.helpers import flat, kron_laplacian

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")

SHAPES = [(1, 1), (1, 7), (7, 1), (2, 2), (3, 5), (16, 9), (33, 64)]


def test_impulse_response_is_printed_mask():
    mask = np.loadtxt(os.path.join(GOLDEN, "stencil_mask.txt"))
    x = np.zeros((7, 8))
    x[3, 4] = 1.0
    y = oracle.lap5_apply(x)
    np.testing.assert_array_equal(y[2:5, 3:6], mask)
    y[2:5, 3:6] = 0.0
    assert not y.any()


@pytest.mark.parametrize("nx,ny", SHAPES)
@pytest.mark.parametrize("pad", [0, 3])
def test_matches_kron_sum_exactly_on_integers(nx, ny, pad):
    # Integer inputs make every add order exact, so bit-equality is meaningful.
    rng = np.random.default_rng(nx * 131 + ny)
    x = np.zeros((ny, nx + pad))
    x[:, :nx] = rng.integers(-1000, 1001, size=(ny, nx))
    x[:, nx:] = 7.0  # padding must be ignored
    y = oracle.lap5_apply(x, nx=nx)
    ref = kron_laplacian(nx, ny) @ flat(x, nx)
    np.testing.assert_array_equal(flat(y, nx), ref)
    assert not y[:, nx:].any()


@pytest.mark.parametrize("nx,ny", SHAPES)
def test_matches_kron_sum_on_reals(nx, ny):
    x = gen.uniform_rhs(nx, ny, seed=nx + 17 * ny)
    y = oracle.lap5_apply(x)
    ref = kron_laplacian(nx, ny) @ flat(x, nx)
    bound = 8 * np.finfo(np.float64).eps * (kron_laplacian(nx, ny).__abs__() @ np.abs(flat(x, nx)))
    assert np.all(np.abs(flat(y, nx) - ref) <= bound)


@pytest.mark.parametrize("nx,ny,k,l", [(16, 16, 1, 1), (16, 16, 3, 7), (20, 11, 20, 11), (5, 9, 2, 4)])
def test_closed_form_eigenpairs(nx, ny, k, l):
    v = gen.sine_mode(nx, ny, k, l)
    lam = gen.mode_eigenvalue(nx, ny, k, l)
    y = oracle.lap5_apply(v)
    err = np.abs(y - lam * v).max()
    assert err <= 1e-14 * 8


def test_eigenvalue_extremes_match_sparse_eigensolver():
    import scipy.sparse.linalg as sla
    nx, ny = 12, 9
    A = kron_laplacian(nx, ny).toarray()
    ev = np.linalg.eigvalsh(A)
    closed = sorted(gen.mode_eigenvalue(nx, ny, k, l) for k in range(1, nx + 1) for l in range(1, ny + 1))
    np.testing.assert_allclose(ev, closed, rtol=0, atol=1e-12)
    # and the oracle's stencil operator has the same spectrum (power iteration on lambda_max)
    v = gen.uniform_rhs(nx, ny, seed=3)
    for _ in range(2000):
        v = oracle.lap5_apply(v)
        v /= np.linalg.norm(v)
    lam_max = float(np.vdot(v, oracle.lap5_apply(v)))
    assert abs(lam_max - closed[-1]) < 1e-8
    del sla


@pytest.mark.parametrize("nx,ny", [(1, 1), (3, 5), (31, 17), (64, 64)])
def test_f32_stencil_rounding(nx, ny):
    x64 = gen.uniform_rhs(nx, ny, seed=5 + nx)
    x32 = x64.astype(np.float32)
    y32 = oracle.lap5_apply(x32, dtype=np.float32)
    exact = oracle.lap5_apply(x32.astype(np.float64))  # exact-ish: float inputs, double sums
    absb = np.abs(kron_laplacian(nx, ny)) @ np.abs(flat(x32.astype(np.float64), nx))
    u = np.finfo(np.float32).eps / 2
    assert np.all(np.abs(flat(y32, nx).astype(np.float64) - flat(exact, nx)) <= 5 * u * absb)
    # integer-valued binary32 inputs are exact
    xi = np.random.default_rng(1).integers(-100, 101, size=(ny, nx)).astype(np.float32)
    np.testing.assert_array_equal(oracle.lap5_apply(xi, dtype=np.float32),
                                  (kron_laplacian(nx, ny) @ xi.reshape(-1).astype(np.float64)).reshape(ny, nx))


def test_bf16_rounding_matches_torch_and_ties():
    rng = np.random.default_rng(11)
    v = np.concatenate([rng.uniform(-4, 4, 5000), rng.standard_normal(5000) * 1e-20,
                        [0.0, -0.0, 1.0, 1 + 2 ** -8, 1 + 3 * 2 ** -8, 1 + 2 ** -8 + 2 ** -20,
                         3.3895314e38, np.inf, -np.inf]]).astype(np.float32)
    bits = oracle.f32_to_bf16_bits(v)
    ref = torch.from_numpy(v).to(torch.bfloat16).view(torch.int16).numpy().view(np.uint16)
    np.testing.assert_array_equal(bits, ref)
    # ties to even, written out: 1 + 2^-8 is halfway between 1 and 1 + 2^-7 -> 1.0
    assert oracle.bf16_bits_to_f32(oracle.f32_to_bf16_bits(np.float32(1 + 2 ** -8))) == 1.0
    assert oracle.bf16_bits_to_f32(oracle.f32_to_bf16_bits(np.float32(1 + 3 * 2 ** -8))) == 1 + 2 ** -6
    nan = oracle.bf16_bits_to_f32(oracle.f32_to_bf16_bits(np.float32(np.nan)))
    assert math.isnan(float(nan))


@pytest.mark.parametrize("nx,ny", [(1, 1), (8, 3), (40, 40)])
def test_bf16_stencil(nx, ny):
    rng = np.random.default_rng(nx)
    # small integers are exact in bf16 and every binary32 sum of them is exact
    xi = rng.integers(-60, 61, size=(ny, nx)).astype(np.float32)
    y = oracle.lap5_apply(oracle.f32_to_bf16_bits(xi), dtype="bf16")
    exact = (kron_laplacian(nx, ny) @ xi.reshape(-1).astype(np.float64)).astype(np.float32)
    np.testing.assert_array_equal(y.reshape(-1), oracle.f32_to_bf16_bits(exact))
    # real-valued inputs: within one bf16 rounding of the binary64 result
    xr = oracle.bf16_bits_to_f32(oracle.f32_to_bf16_bits(gen.uniform_rhs(nx, ny, seed=9).astype(np.float32)))
    yr = oracle.bf16_bits_to_f32(oracle.lap5_apply(oracle.f32_to_bf16_bits(xr), dtype="bf16")).astype(np.float64)
    ex = (kron_laplacian(nx, ny) @ xr.reshape(-1).astype(np.float64)).reshape(ny, nx)
    absb = (np.abs(kron_laplacian(nx, ny)) @ np.abs(xr.reshape(-1).astype(np.float64))).reshape(ny, nx)
    assert np.all(np.abs(yr - ex) <= 2.0 ** -8 * np.abs(ex) + 6 * 2.0 ** -24 * absb)
