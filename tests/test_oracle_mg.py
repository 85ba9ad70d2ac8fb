"""Pins for the oracle's multigrid-preconditioned CG (Algorithm 1 with
M^-1 = one geometric V-cycle) and its pipelined form (Algorithm 2 with M).

References independent of the oracle: dense transfer matrices built column by
column (restriction = transpose of prolongation), exact interpolation of
bilinear functions, dense Cholesky and sparse direct solves, symmetry and
positive definiteness of M^-1 probed with random vectors, the V-cycle's
contraction as a stationary iteration (textbook range for damped-Jacobi
V(2,2) on the model problem), size-independent iteration counts, and the
identity preconditioner reproducing classic CG (and, pipelined, Algorithm 2)
bit for bit, the pipelined form tracking the classic one.  Planted mistakes
in a temporary copy of the oracle are each caught.
"""
import os
import subprocess

import numpy as np
import pytest
import scipy.linalg as sla
import scipy.sparse.linalg as spla

import lap5_inputs as gen
import oracle
from tests.helpers import flat, kron_laplacian, unflat


def _dense_P(nx, ny):
    nyc, nxc = oracle.mg_coarse_shape(ny, nx)
    cols = []
    for k in range(nxc * nyc):
        e = np.zeros(nxc * nyc)
        e[k] = 1.0
        cols.append(oracle.mg_prolong_add(e.reshape(nyc, nxc), np.zeros((ny, nx))).reshape(-1))
    return np.array(cols).T


def _dense_R(nx, ny):
    rows = []
    for k in range(nx * ny):
        e = np.zeros(nx * ny)
        e[k] = 1.0
        rows.append(oracle.mg_restrict(e.reshape(ny, nx)).reshape(-1))
    return np.array(rows).T


@pytest.mark.parametrize("nx,ny", [(7, 5), (8, 6), (9, 9), (4, 3), (3, 8)])
def test_restriction_is_transpose_of_prolongation(nx, ny):
    P, R = _dense_P(nx, ny), _dense_R(nx, ny)
    assert np.array_equal(R, P.T)
    # P's weights: 1 at coincident points, 1/2 and 1/4 between
    assert set(np.unique(P)) <= {0.0, 0.25, 0.5, 1.0}


@pytest.mark.parametrize("nx,ny", [(15, 11), (16, 12), (31, 31)])
def test_prolongation_reproduces_bilinear_functions(nx, ny):
    f = lambda i, j: 1.0 + 2.0 * i - 3.0 * j + 0.5 * i * j  # noqa: E731 -- bilinear in fine index coordinates
    nyc, nxc = oracle.mg_coarse_shape(ny, nx)
    J, I = np.mgrid[0:nyc, 0:nxc]
    ec = f(2 * I + 1, 2 * J + 1).astype(np.float64)
    x = oracle.mg_prolong_add(ec, np.zeros((ny, nx)))
    jj, ii = np.mgrid[0:ny, 0:nx]
    # exact wherever every coarse point the interpolation uses exists
    inside = (ii >= 1) & (ii <= 2 * nxc - 1) & (jj >= 1) & (jj <= 2 * nyc - 1)
    assert np.array_equal(x[inside], f(ii, jj)[inside])


def test_restriction_of_constant_is_four_in_the_interior():
    nx, ny = 13, 9
    bc = oracle.mg_restrict(np.ones((ny, nx)))
    assert np.all(bc == 4.0)  # (1+2+1+2+4+2+1+2+1)/4; every 3x3 patch is inside for odd sizes


@pytest.mark.parametrize("nx,ny", [(31, 31), (40, 23), (64, 64), (1, 9)])
def test_preconditioner_is_symmetric_positive_definite(nx, ny):
    rng = np.random.default_rng(nx * ny)
    for _ in range(5):
        u, v = rng.standard_normal((ny, nx)), rng.standard_normal((ny, nx))
        Mu, Mv = oracle.mg_precond(u), oracle.mg_precond(v)
        s1, s2 = float(np.vdot(u, Mv)), float(np.vdot(Mu, v))
        assert abs(s1 - s2) <= 1e-13 * (np.linalg.norm(u) * np.linalg.norm(Mv))
        assert float(np.vdot(v, Mv)) > 0.0


@pytest.mark.parametrize("n", [31, 63])
def test_vcycle_contraction_in_textbook_range(n):
    # error propagation E = I - M^-1 A; damped-Jacobi V(2,2) on the model
    # problem contracts by roughly 0.1 per cycle; power iteration on E
    A = kron_laplacian(n, n)
    rng = np.random.default_rng(1)
    e = rng.standard_normal(n * n)
    rho = 0.0
    for _ in range(40):
        e_new = e - flat(oracle.mg_precond((A @ e).reshape(n, n)), n)
        rho = np.linalg.norm(e_new) / np.linalg.norm(e)
        e = e_new / np.linalg.norm(e_new)
    assert 0.02 < rho < 0.2, rho


@pytest.mark.parametrize("nx,ny", [(2, 2), (3, 5), (16, 16), (16, 7), (1, 12)])
def test_pcg_matches_dense_cholesky(nx, ny):
    A = kron_laplacian(nx, ny).toarray()
    b = gen.uniform_rhs(nx, ny, seed=nx * 100 + ny)
    x_ref = sla.cho_solve(sla.cho_factor(A), flat(b, nx))
    x, info = oracle.cg_pcg(b, tol=1e-13, maxit=200)
    assert info["status"] == oracle.OK
    err = np.linalg.norm(flat(x, nx) - x_ref) / np.linalg.norm(x_ref)
    assert err <= gen.condition_number(nx, ny) * 1e-13 * 4


def test_pcg_matches_sparse_direct_solve_on_pitched_grid():
    nx, ny = 100, 83
    b = gen.uniform_rhs(nx, ny, seed=8, ld=gen.pitch(nx, 8))
    x_ref = spla.spsolve(kron_laplacian(nx, ny).tocsc(), flat(b, nx))
    x, info = oracle.cg_pcg(b, tol=1e-12, maxit=200, nx=nx)
    assert info["status"] == oracle.OK and info["relres_true"] <= 1.5e-12
    assert np.linalg.norm(flat(x, nx) - x_ref) <= gen.condition_number(nx, ny) * 2e-12 * np.linalg.norm(x_ref)
    assert not x[:, nx:].any()


def test_iteration_counts_do_not_grow_with_the_grid():
    its = {}
    for n in (15, 31, 63, 127, 255, 64, 128, 256):
        b = gen.uniform_rhs(n, n, seed=n)
        _, info = oracle.cg_pcg(b, tol=1e-10, maxit=200)
        assert info["status"] == oracle.OK
        its[n] = info["iters"]
    nested = [its[n] for n in (15, 31, 63, 127, 255)]
    assert max(nested) <= 10 and max(nested) - min(nested) <= 1, its
    assert max(its[n] for n in (64, 128, 256)) <= 20, its
    # plain CG needs hundreds of iterations at 255^2
    _, info = oracle.cg_classic(gen.uniform_rhs(255, 255, seed=255), tol=1e-10, maxit=5000)
    assert info["iters"] > 20 * its[255]


def test_identity_preconditioner_reproduces_classic_cg():
    b = gen.uniform_rhs(40, 33, seed=2)
    x1, i1 = oracle.cg_pcg(b, tol=0.0, maxit=25, levels=0)
    x2, i2 = oracle.cg_classic(b, tol=0.0, maxit=25)
    assert np.array_equal(x1, x2) and i1["iters"] == i2["iters"] == 25


def test_pipelined_pcg_with_identity_is_algorithm_2():
    # M = I turns the preconditioned recurrences into Algorithm 2 line by line
    b = gen.uniform_rhs(40, 33, seed=2)
    x1, i1 = oracle.cg_ppcg(b, tol=0.0, maxit=25, levels=0)
    x2, i2 = oracle.cg_newcg(b, tol=0.0, maxit=25)
    assert np.array_equal(x1, x2) and i1["iters"] == i2["iters"] == 25


@pytest.mark.parametrize("nx,ny", [(63, 63), (100, 83), (300, 200)])
def test_pipelined_pcg_tracks_pcg(nx, ny):
    # the same Krylov iterates in exact arithmetic; early iterations agree to rounding
    b = gen.uniform_rhs(nx, ny, seed=nx + ny)
    for k in (1, 4, 8):
        x1, i1 = oracle.cg_ppcg(b, tol=0.0, maxit=k)
        x2, i2 = oracle.cg_pcg(b, tol=0.0, maxit=k)
        assert i1["iters"] == i2["iters"] == k
        assert np.linalg.norm(x1 - x2) <= 1e-10 * np.linalg.norm(x2)
    x, info = oracle.cg_ppcg(b, tol=1e-10, maxit=200)
    _, ic = oracle.cg_pcg(b, tol=1e-10, maxit=200)
    assert info["status"] == oracle.OK and abs(info["iters"] - ic["iters"]) <= 1


@pytest.mark.parametrize("nx,ny", [(3, 5), (16, 7)])
def test_pipelined_pcg_matches_dense_cholesky(nx, ny):
    A = kron_laplacian(nx, ny).toarray()
    b = gen.uniform_rhs(nx, ny, seed=nx * 100 + ny)
    x_ref = sla.cho_solve(sla.cho_factor(A), flat(b, nx))
    x, info = oracle.cg_ppcg(b, tol=1e-13, maxit=200)
    assert info["status"] == oracle.OK
    assert np.linalg.norm(flat(x, nx) - x_ref) <= gen.condition_number(nx, ny) * 4e-13 * np.linalg.norm(x_ref)


def test_pcg_a_norm_error_is_monotone():
    n = 40
    A = kron_laplacian(n, n)
    b = gen.uniform_rhs(n, n, seed=3)
    x_ref = spla.spsolve(A.tocsc(), flat(b, n))
    errs = []
    for k in range(1, 10):
        x, _ = oracle.cg_pcg(b, tol=0.0, maxit=k)
        e = flat(x, n) - x_ref
        errs.append(float(e @ (A @ e)))
    assert all(e2 <= e1 * (1 + 1e-9) for e1, e2 in zip(errs, errs[1:])), errs


# --------------------------------------------------------------------------
# Planted mistakes (compiled from temporary copies of the oracle source)
# --------------------------------------------------------------------------
SRC = os.path.join(os.path.dirname(oracle.__file__), "lap5_oracle.c")
MUTATIONS = {
    "restrict_edge_weight": ("const double s1 = ((mg_at(r, nx, ny, i - 1, j) + mg_at(r, nx, ny, i + 1, j)) + "
                             "mg_at(r, nx, ny, i, j - 1)) +",
                             "const double s1 = ((mg_at(r, nx, ny, i - 1, j) + mg_at(r, nx, ny, i + 2, j)) + "
                             "mg_at(r, nx, ny, i, j - 1)) +"),
    "prolong_half_weight": ("v = 0.5 * (mg_at(ec, nxc, nyc, I - 1, J) + mg_at(ec, nxc, nyc, I, J));",
                            "v = 0.25 * (mg_at(ec, nxc, nyc, I - 1, J) + mg_at(ec, nxc, nyc, I, J));"),
    "jacobi_sign": ("xo[t] = xi[t] + ORA_MG_C * (b[t] - tmp[t]);", "xo[t] = xi[t] - ORA_MG_C * (b[t] - tmp[t]);"),
    "pcg_beta_uses_rr": ("double beta = gnew / gamma;\n    gamma = gnew;\n    xpby64(nx, ny, ld, z, beta, p);",
                         "double beta = rr / gamma;\n    gamma = gnew;\n    xpby64(nx, ny, ld, z, beta, p);"),
    "ppcg_r_uses_q": ("axpy64(nx, ny, ld, r, -alpha, s);                    /* r = r - alpha s */",
                      "axpy64(nx, ny, ld, r, -alpha, q);                    /* r = r - alpha s */"),
    "ppcg_q_drops_beta": ("xpby64(nx, ny, ld, m, beta, q);                    /* q = m + beta q */",
                          "xpby64(nx, ny, ld, m, 0.0, q);                    /* q = m + beta q */"),
    "pcg_p_from_r": ("xpby64(nx, ny, ld, z, beta, p);                      /* p = z + beta p */",
                     "xpby64(nx, ny, ld, r, beta, p);                      /* p = z + beta p */"),
}


def _mg_pins_pass():
    try:
        P, R = _dense_P(7, 5), _dense_R(7, 5)
        if not np.array_equal(R, P.T):
            return False
        rng = np.random.default_rng(0)
        u, v = rng.standard_normal((31, 31)), rng.standard_normal((31, 31))
        Mu, Mv = oracle.mg_precond(u), oracle.mg_precond(v)
        if abs(np.vdot(u, Mv) - np.vdot(Mu, v)) > 1e-13 * np.linalg.norm(u) * np.linalg.norm(Mv):
            return False
        n = 31
        A = kron_laplacian(n, n)
        e = rng.standard_normal(n * n)
        for _ in range(20):
            e_new = e - flat(oracle.mg_precond((A @ e).reshape(n, n)), n)
            rho = np.linalg.norm(e_new) / np.linalg.norm(e)
            e = e_new / np.linalg.norm(e_new)
        if not rho < 0.2:
            return False
        b = gen.uniform_rhs(16, 7, seed=3)
        x_ref = sla.cho_solve(sla.cho_factor(kron_laplacian(16, 7).toarray()), flat(b, 16))
        x, info = oracle.cg_pcg(b, tol=1e-12, maxit=100)
        if info["status"] != oracle.OK or np.linalg.norm(flat(x, 16) - x_ref) > 1e-9 * np.linalg.norm(x_ref):
            return False
        _, info = oracle.cg_pcg(gen.uniform_rhs(63, 63, seed=6), tol=1e-10, maxit=200)
        if not (info["status"] == oracle.OK and info["iters"] <= 10):
            return False
        b = gen.uniform_rhs(63, 63, seed=7)
        x1, _ = oracle.cg_ppcg(b, tol=0.0, maxit=6)
        x2, _ = oracle.cg_pcg(b, tol=0.0, maxit=6)
        return bool(np.all(np.isfinite(x1))) and np.linalg.norm(x1 - x2) <= 1e-10 * np.linalg.norm(x2)
    except Exception:
        return False


def test_unmutated_oracle_passes_mg_pins():
    assert _mg_pins_pass()


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_planted_mg_mistake_is_caught(name, tmp_path):
    src = open(SRC).read()
    old, new = MUTATIONS[name]
    assert src.count(old) == 1, name
    path_c, path_so = str(tmp_path / (name + ".c")), str(tmp_path / (name + ".so"))
    with open(path_c, "w") as f:
        f.write(src.replace(old, new))
    subprocess.run(["gcc", "-O1", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared", "-o", path_so, path_c, "-lm"],
                   check=True)
    saved = oracle._lib
    real_build = oracle._build.build
    try:
        oracle._lib = None
        oracle._build.build = lambda force=False: path_so
        oracle.lib()
        caught = not _mg_pins_pass()
    finally:
        oracle._build.build = real_build
        oracle._lib = saved
    assert caught, "pins did not catch the planted mistake " + name
