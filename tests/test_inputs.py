"""The seeded input recipe (the stand-in for the paper's N x N workloads):
each generator gives what its description says, deterministically per seed,
with zero padding columns.  The manufactured right-hand side is checked
against the oracle's stencil, which the generator does not use."""
import math

import numpy as np
import pytest

import lap5_inputs as gen
import oracle


def test_uniform_rhs_range_padding_and_seeding():
    b = gen.uniform_rhs(300, 200, seed=7, ld=304)
    assert b.shape == (200, 304) and b.dtype == np.float64
    core = b[:, :300]
    assert core.min() >= -1.0 and core.max() < 1.0
    assert not b[:, 300:].any()
    assert abs(core.mean()) < 0.01 and abs(core.var() - 1.0 / 3.0) < 0.01  # U[-1,1): mean 0, variance 1/3
    np.testing.assert_array_equal(b, gen.uniform_rhs(300, 200, seed=7, ld=304))
    assert not np.array_equal(core, gen.uniform_rhs(300, 200, seed=8)[:, :300])
    # the padded and unpadded draws are the same numbers
    np.testing.assert_array_equal(core, gen.uniform_rhs(300, 200, seed=7))


def test_gaussian_field_moments():
    g = gen.gaussian_field(512, 512, seed=3, ld=520)
    core = g[:, :512]
    assert abs(core.mean()) < 0.01 and abs(core.std() - 1.0) < 0.01
    assert not g[:, 512:].any()


@pytest.mark.parametrize("nx,ny", [(33, 65), (127, 40), (256, 256)])
def test_manufactured_rhs_is_A_ustar_plus_noise(nx, ny):
    noise = 1e-3
    b = gen.manufactured_rhs(nx, ny, seed=2, noise=noise)
    u = gen.sine_mode(nx, ny, 1, 1)
    au = oracle.lap5_apply(u)  # the stencil, applied by the oracle
    xi = (b - au) / noise
    # what is left is the standard normal noise of the seed (A u* = lambda_11 u* up to rounding)
    rng = np.random.default_rng(2)
    np.testing.assert_allclose(xi, rng.standard_normal((ny, nx)), rtol=0, atol=1e-9)
    # without noise b is A u* to the rounding of a stencil of O(1) values (the
    # result itself is O(h^2), so the bound is absolute)
    b0 = gen.manufactured_rhs(nx, ny, seed=2, noise=0.0)
    np.testing.assert_allclose(b0, au, rtol=0, atol=1e-14)


def test_sine_mode_is_the_closed_form_eigenvector():
    nx, ny = 40, 25
    for k, l in ((1, 1), (3, 2), (40, 25)):
        v = gen.sine_mode(nx, ny, k, l)
        lam = gen.mode_eigenvalue(nx, ny, k, l)
        np.testing.assert_allclose(oracle.lap5_apply(v), lam * v, rtol=0, atol=1e-13)
    # condition number: largest over smallest eigenvalue of the closed form
    h = math.pi / (2 * (nx + 1))
    assert gen.condition_number(nx, nx) == pytest.approx(1.0 / math.tan(h) ** 2, rel=1e-12)


def test_batched_shapes_and_rhs():
    nxs, nys = gen.batched_shapes(256, 64, 1024, seed=4)
    assert len(nxs) == len(nys) == 256
    assert min(nxs + nys) >= 64 and max(nxs + nys) <= 1024
    assert abs(np.mean(nxs + nys) - 544) < 30  # uniform on {64..1024}: mean 544
    assert (nxs, nys) == gen.batched_shapes(256, 64, 1024, seed=4)
    bs = gen.batched_rhs(nxs[:5], nys[:5], seed=4, elem_bytes=8, align_bytes=32)
    for (nx, ny, b) in zip(nxs, nys, bs):
        assert b.shape[0] == ny and b.shape[1] >= nx and (b.shape[1] * 8) % 32 == 0
        assert not b[:, nx:].any()


def test_pitch():
    for nx in (1, 3, 4, 100, 101, 1030):
        for es, al in ((8, 16), (4, 16), (8, 32), (2, 16)):
            ld = gen.pitch(nx, es, al)
            assert ld >= nx and (ld * es) % al == 0 and ld - nx < al // es


def test_rel_err_sees_a_single_wrong_point():
    # the GPU parity tests compare with the larger of the norm-wise and the
    # element-wise relative difference
    from tests.helpers import rel_err
    b = np.ones(4096 * 4096 // 64)
    a = b.copy()
    a[123] += 1e-7
    assert np.linalg.norm(a - b) / np.linalg.norm(b) < 2e-10  # a norm averages it away
    assert rel_err(a, b) >= 1e-7
    assert rel_err(b, b) == 0.0 and rel_err(np.zeros(3), np.zeros(3)) == 0.0
