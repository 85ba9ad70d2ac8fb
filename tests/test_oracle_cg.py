"""Pins for the oracle's Algorithm 1 (classic CG) and Algorithm 2 (NewCG).

The references are independent of the oracle: dense Cholesky and banded
(Thomas) solves from scipy, a sparse direct solve, exact rational arithmetic,
closed-form eigenpairs, and the textbook CG invariants (A-orthogonal search
directions, orthogonal residuals, monotone A-norm error within the Chebyshev
bound, termination in as many steps as the right-hand side has distinct
eigenvalues).
"""
import math
import os
from fractions import Fraction

import numpy as np
import pytest
import scipy.linalg as sla
import scipy.sparse.linalg as spla

import lap5_inputs as gen
import oracle
from tests.helpers import flat, kron_laplacian, unflat

VARIANTS = ["classic", "newcg"]
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def solve(b, variant, **kw):
    return oracle.cg_solve(b, variant=variant, **kw)


@pytest.mark.parametrize("variant", VARIANTS)
@pytest.mark.parametrize("nx,ny", [(2, 2), (3, 5), (8, 8), (16, 16), (16, 7)])
def test_dense_cholesky(variant, nx, ny):
    A = kron_laplacian(nx, ny).toarray()
    b = gen.uniform_rhs(nx, ny, seed=nx * 100 + ny)
    x_ref = sla.cho_solve(sla.cho_factor(A), flat(b, nx))
    x, info = solve(b, variant, tol=1e-13, maxit=10 * nx * ny)
    assert info["status"] == oracle.OK
    kappa = gen.condition_number(nx, ny)
    err = np.linalg.norm(flat(x, nx) - x_ref) / np.linalg.norm(x_ref)
    assert err <= kappa * 1e-13 * 2
    assert info["relres_true"] <= 2e-13


@pytest.mark.parametrize("variant", VARIANTS)
@pytest.mark.parametrize("nx,ny", [(50, 1), (1, 37)])
def test_one_row_is_tridiagonal_thomas(variant, nx, ny):
    n = max(nx, ny)
    b = gen.uniform_rhs(nx, ny, seed=n)
    ab = np.zeros((3, n))
    ab[0, 1:] = -1.0
    ab[1, :] = 4.0
    ab[2, :-1] = -1.0
    x_ref = sla.solve_banded((1, 1), ab, flat(b, nx))
    x, info = solve(b, variant, tol=1e-14, maxit=500)
    assert info["status"] == oracle.OK
    np.testing.assert_allclose(flat(x, nx), x_ref, rtol=0, atol=1e-13 * np.abs(x_ref).max())


@pytest.mark.parametrize("variant", VARIANTS)
def test_single_point(variant):
    b = np.array([[3.0]])
    x, info = solve(b, variant, tol=1e-12, maxit=10)
    assert info["status"] == oracle.OK and info["iters"] == 1
    assert x[0, 0] == 0.75


def _exact_cg_iterations(nx, ny, b_int):
    """Algorithm 1 in exact rational arithmetic; returns the number of steps to r = 0."""
    A = kron_laplacian(nx, ny).toarray().astype(int)
    n = nx * ny
    x = [Fraction(0)] * n
    r = [Fraction(int(v)) for v in b_int]
    p = list(r)
    g = sum(v * v for v in r)
    k = 0
    while g != 0:
        z = [sum(Fraction(int(A[i, j])) * p[j] for j in range(n) if A[i, j]) for i in range(n)]
        a = g / sum(zi * pi for zi, pi in zip(z, p))
        x = [xi + a * pi for xi, pi in zip(x, p)]
        r = [ri - a * zi for ri, zi in zip(r, z)]
        gn = sum(v * v for v in r)
        k += 1
        p = [ri + (gn / g) * pi for ri, pi in zip(r, p)]
        g = gn
    return k, x


def test_exact_rational_2x2():
    # A = [[4,-1,-1,0],[-1,4,0,-1],[-1,0,4,-1],[0,-1,-1,4]] has eigenvalues 2, 4, 4, 6
    k, x_exact = _exact_cg_iterations(2, 2, [1, 0, 0, 0])
    assert k == 3
    for variant in VARIANTS:
        x, info = solve(np.array([[1.0, 0.0], [0.0, 0.0]]), variant, tol=1e-15, maxit=10)
        assert info["iters"] <= 3
        np.testing.assert_allclose(flat(x, 2), [float(v) for v in x_exact], rtol=1e-15, atol=1e-16)
    # x_exact = A^{-1} e_1 = (7/24, 1/12, 1/12, 1/24)
    assert x_exact == [Fraction(7, 24), Fraction(1, 12), Fraction(1, 12), Fraction(1, 24)]


@pytest.mark.parametrize("variant", VARIANTS)
def test_eigvec_rhs_terminates_in_one_step(variant):
    nx = ny = 64
    lam = gen.mode_eigenvalue(nx, ny, 1, 1)
    u = gen.sine_mode(nx, ny, 1, 1)
    b = lam * u  # the manufactured right-hand side without noise
    tr = oracle.Trace(ny, nx, 2, 5, newcg=(variant == "newcg"))
    x, info = solve(b, variant, tol=1e-12, maxit=5, trace=tr)
    assert info["iters"] == 1 and info["status"] == oracle.OK
    assert abs(tr.alpha[0] - 1.0 / lam) <= 1e-13 / lam
    assert np.abs(x - u).max() <= 1e-13


@pytest.mark.parametrize("variant", VARIANTS)
def test_m_distinct_eigenvalues_terminate_in_m_steps(variant):
    nx, ny = 24, 20
    modes = [(1, 1), (2, 3), (5, 1), (7, 9)]
    b = sum((m + 1.0) * gen.sine_mode(nx, ny, k, l) for m, (k, l) in enumerate(modes))
    tr = oracle.Trace(ny, nx, 1, 10, newcg=(variant == "newcg"))
    x, info = solve(b, variant, tol=0.0, maxit=len(modes), trace=tr)
    # exact arithmetic gives r = 0 at step m; rounding leaves ~1e-11 here
    assert tr.relres[len(modes) - 1] > 1e-4
    assert tr.relres[len(modes)] < 1e-9
    x_ref = sum((m + 1.0) / gen.mode_eigenvalue(nx, ny, k, l) * gen.sine_mode(nx, ny, k, l)
                for m, (k, l) in enumerate(modes))
    assert np.abs(x - x_ref).max() <= 1e-9 * np.abs(x_ref).max()


def test_classic_orthogonality_invariants():
    nx = ny = 32
    A = kron_laplacian(nx, ny)
    b = gen.uniform_rhs(nx, ny, seed=7)
    K = 20
    tr = oracle.Trace(ny, nx, K + 1, K)
    oracle.cg_classic(b, tol=0.0, maxit=K, trace=tr)
    P = tr.p[:K].reshape(K, -1)
    R = tr.r[:K].reshape(K, -1)
    AP = (A @ P.T).T
    G = P @ AP.T
    d = np.sqrt(np.diag(G))
    Gn = np.abs(G) / np.outer(d, d)
    RR = np.abs(R @ R.T) / np.outer(np.linalg.norm(R, axis=1), np.linalg.norm(R, axis=1))
    off = ~np.eye(K, dtype=bool)
    assert Gn[off].max() <= 1e-8
    assert RR[off].max() <= 1e-8


@pytest.mark.parametrize("variant", VARIANTS)
def test_a_norm_error_monotone_and_chebyshev_bound(variant):
    nx = ny = 32
    A = kron_laplacian(nx, ny)
    b = gen.uniform_rhs(nx, ny, seed=8)
    x_star = spla.spsolve(A.tocsc(), flat(b, nx))
    K = 60
    tr = oracle.Trace(ny, nx, K + 1, K, newcg=(variant == "newcg"))
    solve(b, variant, tol=0.0, maxit=K, trace=tr)
    kappa = gen.condition_number(nx, ny)
    rho = (math.sqrt(kappa) - 1) / (math.sqrt(kappa) + 1)
    errs = []
    for k in range(K + 1):
        e = tr.x[k].reshape(-1) - x_star
        errs.append(math.sqrt(float(e @ (A @ e))))
    for k in range(1, K + 1):
        assert errs[k] <= errs[k - 1] * (1 + 1e-10)
        assert errs[k] <= 2 * rho ** k * errs[0] * (1 + 1e-9)


@pytest.mark.parametrize("n,kmax", [(32, 30), (100, 30)])
def test_newcg_iterates_equal_classic(n, kmax):
    b = gen.uniform_rhs(n, n, seed=n)
    tc = oracle.Trace(n, n, kmax + 1, kmax)
    tn = oracle.Trace(n, n, kmax + 1, kmax, newcg=True)
    oracle.cg_classic(b, tol=0.0, maxit=kmax, trace=tc)
    oracle.cg_newcg(b, tol=0.0, maxit=kmax, trace=tn)
    for k in range(1, kmax + 1):
        rel = np.linalg.norm(tc.x[k] - tn.x[k]) / np.linalg.norm(tc.x[k])
        assert rel <= 1e-10, (k, rel)
    np.testing.assert_allclose(tn.alpha[:kmax], tc.alpha[:kmax], rtol=1e-9)
    np.testing.assert_allclose(tn.beta[1:kmax], tc.beta[1:kmax], rtol=1e-8)


@pytest.mark.parametrize("n,kmax", [(32, 30), (100, 30)])
def test_newcg_stable_iterates_equal_classic(n, kmax):
    # alpha from (p, A p) = delta + 2 beta (r, q_old) + beta^2 (p_old, q_old):
    # equal to Algorithm 2's (and Algorithm 1's) alpha in exact arithmetic
    b = gen.uniform_rhs(n, n, seed=n + 7)
    tc = oracle.Trace(n, n, kmax + 1, kmax)
    ts = oracle.Trace(n, n, kmax + 1, kmax, newcg=True)
    oracle.cg_classic(b, tol=0.0, maxit=kmax, trace=tc)
    oracle.cg_newcg(b, tol=0.0, maxit=kmax, trace=ts, stable=True)
    for k in range(1, kmax + 1):
        rel = np.linalg.norm(tc.x[k] - ts.x[k]) / np.linalg.norm(tc.x[k])
        assert rel <= 1e-10, (k, rel)
    np.testing.assert_allclose(ts.alpha[:kmax], tc.alpha[:kmax], rtol=1e-9)
    np.testing.assert_allclose(ts.beta[1:kmax], tc.beta[1:kmax], rtol=1e-8)


@pytest.mark.parametrize("nx,ny", [(1, 1), (3, 5), (16, 16), (9, 14)])
def test_newcg_stable_dense_cholesky(nx, ny):
    A = kron_laplacian(nx, ny).toarray()
    b = gen.uniform_rhs(nx, ny, seed=nx * 5 + ny)
    x_ref = sla.cho_solve(sla.cho_factor(A), flat(b, nx))
    x, info = oracle.cg_newcg(b, tol=1e-13, maxit=2000, stable=True)
    assert info["status"] == oracle.OK
    assert np.linalg.norm(flat(x, nx) - x_ref) <= 1e-11 * np.linalg.norm(x_ref) * gen.condition_number(nx, ny)


def test_newcg_stable_survives_the_attainable_accuracy_floor():
    # Near its attainable accuracy Algorithm 2's scalar recurrence for alpha
    # drifts (consecutive residuals are no longer orthogonal) and the
    # iteration breaks down; alpha from the current vectors keeps going down to
    # classic CG's true-residual floor.
    n = 128
    b = gen.manufactured_rhs(n, n, seed=2)
    _, ia = oracle.cg_newcg(b, tol=1e-15, maxit=2000, rr_period=100)
    assert ia["status"] == oracle.ERR_BREAKDOWN
    xs, i_s = oracle.cg_newcg(b, tol=1e-15, maxit=2000, rr_period=100, stable=True)
    _, ic = oracle.cg_classic(b, tol=1e-15, maxit=2000)
    assert i_s["status"] == oracle.NOT_CONVERGED and i_s["iters"] == 2000
    assert i_s["relres_true"] <= 3 * ic["relres_true"] and i_s["relres_true"] <= 1e-11
    # and to a tolerance that Algorithm 2 also meets, the two agree
    x2, i2 = oracle.cg_newcg(b, tol=1e-10, maxit=2000, rr_period=100)
    x3, i3 = oracle.cg_newcg(b, tol=1e-10, maxit=2000, rr_period=100, stable=True)
    assert i2["status"] == i3["status"] == oracle.OK and abs(i2["iters"] - i3["iters"]) <= 2


def test_newcg_auxiliary_identities():
    nx, ny = 40, 24
    A = kron_laplacian(nx, ny)
    b = gen.uniform_rhs(nx, ny, seed=12)
    K = 15
    tn = oracle.Trace(ny, nx, K + 1, K, newcg=True)
    oracle.cg_newcg(b, tol=0.0, maxit=K, trace=tn)
    for k in range(K):
        r, w = tn.r[k].reshape(-1), tn.w[k].reshape(-1)
        p, q, z = tn.p[k].reshape(-1), tn.q[k].reshape(-1), tn.z[k].reshape(-1)
        assert np.linalg.norm(w - A @ r) <= 1e-12 * np.linalg.norm(A @ r) * (k + 1)
        assert np.linalg.norm(q - A @ p) <= 1e-12 * np.linalg.norm(A @ p) * (k + 1)
        assert np.linalg.norm(z - A @ q) <= 1e-12 * np.linalg.norm(A @ q) * (k + 1)


def test_newcg_residual_replacement_keeps_true_residual():
    n = 64
    b = gen.uniform_rhs(n, n, seed=21)
    x_ref = spla.spsolve(kron_laplacian(n, n).tocsc(), flat(b, n))
    x, info = oracle.cg_newcg(b, tol=1e-12, maxit=2000, rr_period=20)
    assert info["status"] == oracle.OK
    assert info["relres_true"] <= 2e-12
    kappa = gen.condition_number(n, n)
    assert np.linalg.norm(flat(x, n) - x_ref) / np.linalg.norm(x_ref) <= kappa * 2e-12


@pytest.mark.parametrize("variant", VARIANTS)
def test_zero_rhs(variant):
    b = np.zeros((5, 6))
    x0 = np.ones((5, 6))
    x, info = solve(b, variant, x0=x0, tol=1e-8, maxit=10)
    assert info["status"] == oracle.OK and info["iters"] == 0 and not x.any()


@pytest.mark.parametrize("variant", VARIANTS)
def test_maxit_and_tol_edges(variant):
    b = gen.uniform_rhs(20, 20, seed=1)
    x, info = solve(b, variant, tol=1e-8, maxit=0)
    assert info["status"] == oracle.NOT_CONVERGED and info["iters"] == 0 and not x.any()
    x, info = solve(b, variant, tol=0.0, maxit=17)
    assert info["status"] == oracle.NOT_CONVERGED and info["iters"] == 17
    x, info = solve(b, variant, tol=-1.0, maxit=9)
    assert info["status"] == oracle.NOT_CONVERGED and info["iters"] == 9


@pytest.mark.parametrize("variant", VARIANTS)
def test_nonfinite_and_invalid(variant):
    b = gen.uniform_rhs(6, 6, seed=1)
    b[2, 3] = np.nan
    x, info = solve(b, variant, tol=1e-8, maxit=10)
    assert info["status"] == oracle.ERR_NONFINITE and not x.any()
    x, info = solve(gen.uniform_rhs(6, 6, seed=1), variant, tol=1e-8, maxit=-1)
    assert info["status"] == oracle.ERR_INVALID_ARG


@pytest.mark.parametrize("variant", VARIANTS)
def test_resume_from_checkpoint(variant):
    # The solver state is x itself: restarting from a saved x continues the solve.
    n = 48
    b = gen.uniform_rhs(n, n, seed=31)
    x_half, info1 = solve(b, variant, tol=0.0, maxit=40)
    x, info2 = solve(b, variant, x0=x_half, tol=1e-11, maxit=2000)
    assert info2["status"] == oracle.OK and info2["relres_true"] <= 2e-11
    x_ref = spla.spsolve(kron_laplacian(n, n).tocsc(), flat(b, n))
    assert np.linalg.norm(flat(x, n) - x_ref) / np.linalg.norm(x_ref) <= gen.condition_number(n, n) * 2e-11


@pytest.mark.parametrize("variant", VARIANTS)
def test_pitched_layout_matches_dense(variant):
    nx, ny, ld = 37, 23, 40
    b = gen.uniform_rhs(nx, ny, seed=4, ld=ld)
    b[:, nx:] = 123.0  # padding garbage must be ignored
    x, info = solve(b, variant, tol=1e-10, maxit=1000, nx=nx)
    x2, info2 = solve(np.ascontiguousarray(b[:, :nx]), variant, tol=1e-10, maxit=1000)
    np.testing.assert_array_equal(x[:, :nx], x2)
    assert info["iters"] == info2["iters"]


def test_paper_iteration_counts_are_reported_only():
    # Context (parity unpinned): the paper's counts for an unstated RHS/tolerance.
    counts = np.loadtxt(os.path.join(GOLDEN, "paper_iteration_counts.txt"))
    for n, paper_iters in counts:
        n = int(n)
        _, info = oracle.cg_classic(gen.uniform_rhs(n, n, seed=1), tol=1e-8, maxit=5000)
        assert info["status"] == oracle.OK
        # a solve from a random RHS needs at least as many steps as the paper's count order of magnitude
        assert info["iters"] > 0 and paper_iters > 0


@pytest.mark.parametrize("inner", ["f32", "bf16pr"])
def test_ir_reaches_fp64_accuracy(inner):
    n = 64
    b = gen.uniform_rhs(n, n, seed=41)
    x_ref = spla.spsolve(kron_laplacian(n, n).tocsc(), flat(b, n))
    x, info = oracle.cg_ir(b, tol=1e-10, inner=inner)
    assert info["status"] == oracle.OK and info["relres_true"] <= 1e-10
    assert info["outer_iters"] >= 2  # one low-precision solve cannot reach 1e-10
    assert np.linalg.norm(flat(x, n) - x_ref) / np.linalg.norm(x_ref) <= gen.condition_number(n, n) * 1e-10


def test_dot2_against_exact_sum():
    rng = np.random.default_rng(5)
    for n in (1000, 200000):
        a = rng.uniform(-1, 1, n).astype(np.float32)
        b = rng.uniform(-1, 1, n).astype(np.float32)
        exact = math.fsum((a.astype(np.float64) * b.astype(np.float64)).tolist())  # products of floats are exact in binary64
        s, c = oracle.dot2_f32(a.reshape(1, -1), b.reshape(1, -1))
        u = 2.0 ** -24
        cond_abs = float(np.abs(a.astype(np.float64) * b.astype(np.float64)).sum())
        assert abs((s + c) - exact) <= 2 * u * abs(exact) + 4 * n * n * u * u * cond_abs
