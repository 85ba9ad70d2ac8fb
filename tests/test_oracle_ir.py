"""Pins of the oracle's mixed-precision path: the inner binary32 / bf16-p,r
classic CG on its own (oracle.inner_cg_f32) and the FP64 refinement loop
around it (oracle.cg_ir).  The refinement is self-correcting, so "reaches
1e-10" alone would not notice a wrong beta, a wrong sign or a missing bf16
rounding; these pins do (tests/test_oracle_mutations.py plants each one).

  * one-step termination on a sine mode (an eigenvector: Algorithm 1 ends
    after one update with d = rin / lambda), binary32;
  * m-step termination on m modes of distinct eigenvalues, binary32;
  * at a fixed iteration count the binary32 iterate stays within a
    rounding-level distance of the binary64 Algorithm 1 on the same data;
  * bf16 p, r: bit-for-bit equality with an independent numpy restatement that
    rounds p and r to bf16 (torch's round-to-nearest-even) after every update,
    takes the Polak-Ribiere beta (r_new, r_new - r_old) / (r_old, r_old) and
    sums with its own Dot2 (TwoProduct from an exact binary64 product, Knuth's
    TwoSum).
"""
import math

import numpy as np
import pytest
import torch

import lap5_inputs as gen
import oracle
from tests.helpers import kron_laplacian

U32 = 2.0 ** -24


def _amplification(n, lams):
    """max over the spectrum of |prod_t (1 - lambda / lambda_t)|: in exact
    arithmetic Algorithm 1 on a combination of the modes lambda_t ends after
    len(lams) updates with that polynomial applied to the residual, so a
    rounding error of the input (~u32 per element) comes out scaled by at most
    this factor."""
    lo, hi = gen.mode_eigenvalue(n, n, 1, 1), gen.mode_eigenvalue(n, n, n, n)
    grid = np.linspace(lo, hi, 20001)
    poly = np.ones_like(grid)
    for lam in lams:
        poly *= 1.0 - grid / lam
    return float(np.max(np.abs(poly)))


@pytest.mark.parametrize("k,l", [(1, 1), (3, 5), (40, 2), (24, 30)])
def test_inner_one_step_on_sine_mode(k, l):
    n = 48
    rin = gen.sine_mode(n, n, k, l).astype(np.float32)
    lam = gen.mode_eigenvalue(n, n, k, l)
    d, r, it, brk = oracle.inner_cg_f32(rin, tol_in=0.0, maxit_in=1, storage="f32")
    assert not brk and it == 1
    ref = rin.astype(np.float64) / lam
    # alpha = (r, r) / (p, A p): the binary32 stencil rounds each of its four
    # subtractions (|error| <= 3 u32 * 8 |p| a point), so (p, A p) = lambda ||p||^2
    # carries a relative error of at most 24 u32 / lambda
    assert np.max(np.abs(d - ref)) <= (16 + 24 / lam) * U32 * np.max(np.abs(ref))
    assert np.linalg.norm(r) <= 4 * U32 * _amplification(n, [lam]) * np.linalg.norm(rin)
    # bf16 p, r: one update moves along p = bf16(rin), within bf16 rounding of rin / lambda
    d1, _, it1, _ = oracle.inner_cg_f32(rin, tol_in=0.0, maxit_in=1, storage="bf16pr")
    assert it1 == 1
    assert np.max(np.abs(d1 - ref)) <= 2.0 ** -8 * np.max(np.abs(ref))


MODES = [(1, 1), (2, 3), (5, 2), (7, 7), (30, 11), (20, 37)]


@pytest.mark.parametrize("first,m", [(0, 2), (0, 3), (0, 4), (4, 2)])
def test_inner_m_modes_terminate_in_m_steps(first, m):
    n = 40
    ks = MODES[first:first + m]
    lams = [gen.mode_eigenvalue(n, n, k, l) for k, l in ks]
    assert len(set(round(x, 12) for x in lams)) == m
    v = sum((0.5 ** t) * gen.sine_mode(n, n, k, l) for t, (k, l) in enumerate(ks))
    rin = v.astype(np.float32)
    d, r, it, brk = oracle.inner_cg_f32(rin, tol_in=0.0, maxit_in=m, storage="f32")
    assert not brk and it == m
    amp = _amplification(n, lams)
    assert np.linalg.norm(r) <= 4 * U32 * amp * np.linalg.norm(rin)
    _, r1, _, _ = oracle.inner_cg_f32(rin, tol_in=0.0, maxit_in=m - 1, storage="f32")
    assert np.linalg.norm(r1) >= 1e-2 * np.linalg.norm(rin)  # not done one step early
    # the solution of A d = rin is sum_t c_t v_t / lambda_t
    ref = sum((0.5 ** t) * gen.sine_mode(n, n, k, l) / lam for t, ((k, l), lam) in enumerate(zip(ks, lams)))
    assert np.linalg.norm(d - ref) <= 4 * U32 * amp / min(lams) * np.linalg.norm(rin) + 16 * U32 * np.linalg.norm(ref)


@pytest.mark.parametrize("k", [5, 25])
def test_inner_f32_tracks_fp64_algorithm1(k):
    # binary32 rounding perturbs each step by ~u32; over k steps on a 64^2 grid
    # (kappa ~ 1.7e3) the iterates stay within ~k * kappa * u32 ~ 3e-3 (a
    # pessimistic bound; measured ~1e-6).  A wrong beta or sign is O(1).
    n = 64
    rin = gen.uniform_rhs(n, n, seed=71).astype(np.float32)
    d, r, it, brk = oracle.inner_cg_f32(rin, tol_in=0.0, maxit_in=k, storage="f32")
    assert it == k and not brk
    x64, info = oracle.cg_classic(rin.astype(np.float64), tol=0.0, maxit=k)
    assert info["iters"] == k
    assert np.linalg.norm(d - x64) <= 1e-4 * np.linalg.norm(x64)
    # the recursive residual tracks the true residual of d to rounding level
    true_r = rin.astype(np.float64) - oracle.lap5_apply(d.astype(np.float64))
    assert np.linalg.norm(r - true_r) <= 1e-5 * np.linalg.norm(rin)


# ---------------------------------------------------------------------------
# independent restatement of the bf16-p,r inner solve
# ---------------------------------------------------------------------------
def _bf16(v):
    return torch.from_numpy(np.ascontiguousarray(v, dtype=np.float32)).to(torch.bfloat16).to(torch.float32).numpy()


def _stencil32(x, nx, ny):
    z = np.zeros((ny + 2, nx + 2), dtype=np.float32)
    z[1:-1, 1:-1] = x[:, :nx]
    c = z[1:-1, 1:-1]
    acc = np.float32(4.0) * c
    acc = acc - z[1:-1, :-2]
    acc = acc - z[1:-1, 2:]
    acc = acc - z[:-2, 1:-1]
    acc = acc - z[2:, 1:-1]
    y = np.zeros_like(x)
    y[:, :nx] = acc
    return y


def _dot2(a, b, nx):
    s = np.float32(0.0)
    c = np.float32(0.0)
    for ai, bi in zip(a[:, :nx].ravel().tolist(), b[:, :nx].ravel().tolist()):
        ai, bi = np.float32(ai), np.float32(bi)
        h = np.float32(ai * bi)
        lo = np.float32(float(ai) * float(bi) - float(h))   # exact: the product error fits binary32
        x = np.float32(s + h)
        z = np.float32(x - s)
        e = np.float32(np.float32(s - np.float32(x - z)) + np.float32(h - z))
        s = x
        c = np.float32(c + np.float32(e + lo))
    return float(s) + float(c)


def _restated_inner(rin, nx, maxit, bf):
    ny = rin.shape[0]
    st = _bf16 if bf else (lambda v: np.asarray(v, dtype=np.float32))
    d = np.zeros_like(rin)
    r = st(rin)
    p = r.copy()
    g = _dot2(r, r, nx)
    k = 0
    while k < maxit and g > 0.0:
        z = _stencil32(p, nx, ny)
        pz = _dot2(p, z, nx)
        a = np.float32(g / pz)
        d = (d + a * p).astype(np.float32)
        r_old = r
        r = st((r - a * z).astype(np.float32))
        gn = _dot2(r, r, nx)
        k += 1
        # bf16 p, r: Polak-Ribiere beta (r_new, r_new - r_old) / (r_old, r_old)
        num = gn - _dot2(r, r_old, nx) if bf else gn
        bt = np.float32(num / g)
        g = gn
        if g <= 0.0:
            break
        p = st((r + bt * p).astype(np.float32))
    return d, r, k


@pytest.mark.parametrize("storage", ["bf16pr", "f32"])
def test_inner_matches_restatement_bit_for_bit(storage):
    nx, ny, ld, k = 23, 17, 24, 30
    rin = gen.uniform_rhs(nx, ny, seed=73, ld=ld).astype(np.float32)
    d, r, it, brk = oracle.inner_cg_f32(rin, tol_in=0.0, maxit_in=k, storage=storage, nx=nx)
    dr, rr, kr = _restated_inner(rin, nx, k, storage == "bf16pr")
    assert it == kr == k and not brk
    np.testing.assert_array_equal(d[:, :nx], dr[:, :nx])
    np.testing.assert_array_equal(r[:, :nx], rr[:, :nx])
    if storage == "bf16pr":  # the stored residual really is bf16
        np.testing.assert_array_equal(r, _bf16(r))


# ---------------------------------------------------------------------------
# the refinement loop, composed from pinned parts
# ---------------------------------------------------------------------------
def _composed_ir(b, nx, max_outer, storage, tol_in, maxit_in):
    """FP64 iterative refinement written out from its definition: r = b - A x
    and (r, r) in binary64 (oracle stencil and index-order dot, both pinned
    elsewhere), r rounded to binary32, the inner solve (pinned above), x += d
    in binary64.  A step whose residual is not below the previous one is kept
    when it lowered the error's energy by at least half of (d, r_old) > 0 --
    (d, r_new) >= -(d, r_old) / 2 (the rule is pinned against the energy's
    definition below) -- and otherwise undone, which ends the solve."""
    x = np.zeros_like(b)
    d, rr_prev, total, outer, reverted, kept = None, None, 0, 0, False, 0
    dro = 0.0
    while True:
        r = b - oracle.lap5_apply(x, nx=nx)
        rr = oracle.dot(r, r, nx=nx)
        if outer > 0 and not rr < rr_prev:
            drn = oracle.dot(d.astype(np.float64), r, nx=nx)
            if dro > 0.0 and drn >= -0.5 * dro:
                kept += 1
            else:
                x = x - d.astype(np.float64)
                reverted = True
                break
        rr_prev = rr
        if outer >= max_outer:
            break
        d, _, k, brk = oracle.inner_cg_f32(r.astype(np.float32), tol_in=tol_in, maxit_in=maxit_in,
                                           storage=storage, nx=nx)
        assert not brk
        total += k
        dro = oracle.dot(d.astype(np.float64), r, nx=nx)
        x = x + d.astype(np.float64)
        outer += 1
    return x, total, outer, reverted, kept


@pytest.mark.parametrize("n,storage,tol_in,maxit_in,max_outer,guard,kept", [
    (40, "f32", 1e-4, 500, 3, False, False),
    (40, "bf16pr", 1e-2, 500, 3, False, False),
    (64, "bf16pr", 1e-2, 20, 6, False, False),
    (64, "bf16pr", 1e-2, 5, 12, False, True),   # truncated inner solves: 2-norm up, energy down
    (96, "bf16pr", 0.5, 10, 12, False, True),
    (64, "f32", 0.0, 384, 6, True, False),      # at the FP64 floor the guard undoes step 4
])
def test_refinement_equals_its_composition(n, storage, tol_in, maxit_in, max_outer, guard, kept):
    b = gen.uniform_rhs(n, n, seed=81)
    x, info = oracle.cg_ir(b, tol=0.0, max_outer=max_outer, inner=storage, tol_in=tol_in, maxit_in=maxit_in)
    xc, total, outer, reverted, nkept = _composed_ir(b, n, max_outer, storage, tol_in, maxit_in)
    assert reverted == guard
    assert (nkept > 0) == kept
    assert info["outer_iters"] == outer and info["iters"] == total
    assert info["status"] == oracle.NOT_CONVERGED
    np.testing.assert_array_equal(x[:, :n], xc[:, :n])
    # an undone step returns the iterate before it: the residual reported is
    # that of the returned x
    if guard:
        assert info["relres_true"] <= info["relres_recursive"] * (1 + 1e-12)


def _energy_cases(n=12, seed=3):
    """Steps d for a residual r_old with known outcomes, from dense algebra:
    d = s e (e = A^-1 r_old), e plus a rough vector that raises the 2-norm but
    hardly the energy, and rough vectors alone."""
    A = kron_laplacian(n, n).toarray()
    rng = np.random.default_rng(seed)
    s1 = np.sin(np.pi * np.arange(1, n + 1) / (n + 1))
    r_old = np.outer(s1, s1).reshape(-1) + 0.05 * rng.standard_normal(n * n)
    e = np.linalg.solve(A, r_old)
    chk = np.indices((n, n)).sum(axis=0) % 2 * 2.0 - 1.0  # the roughest mode's sign pattern
    j = (chk * np.outer(s1, s1)).reshape(-1)
    t = 2.0 * np.linalg.norm(r_old) / np.linalg.norm(A @ j)  # ||A t j|| = 2 ||r_old||
    cases = [s * e for s in (0.3, 0.7, 1.0, 1.4, 1.6, 2.0, 2.5)]
    cases += [e + t * j, e - t * j, e + 3 * t * j, t * j, -t * j, 0.5 * e + 10 * t * j]
    return A, r_old, e, cases


def test_keep_rule_follows_the_energy_definition():
    A, r_old, e, cases = _energy_cases()
    E_old = e @ A @ e
    saw_raised_and_kept = saw_reverted = False
    for d in cases:
        r_new = r_old - A @ d
        rr_old, rr_new = r_old @ r_old, r_new @ r_new
        e_new = e - d
        drop = E_old - e_new @ A @ e_new        # energy removed, from its definition
        claim = d @ r_old
        want = rr_new < rr_old or (claim > 0 and drop >= 0.5 * claim)
        assert abs(drop - 0.5 * claim) > 1e-6 * abs(claim)  # no borderline case
        got = oracle.ir_keep_step(rr_new, rr_old, d @ r_old, d @ r_new)
        assert got == want, (rr_new / rr_old, drop / claim)
        saw_raised_and_kept |= got and rr_new >= rr_old
        saw_reverted |= not got
    assert saw_raised_and_kept and saw_reverted
    # a zero step claims nothing and is undone (the solve would otherwise
    # repeat it until the outer cap)
    assert not oracle.ir_keep_step(r_old @ r_old, r_old @ r_old, 0.0, 0.0)


def test_refinement_contracts_by_the_inner_tolerance():
    # each binary32 refinement step solves A d = r to tol_in (recursive), so
    # the FP64 residual shrinks by about tol_in per step, down to ~1e-10
    n = 64
    b = gen.uniform_rhs(n, n, seed=83)
    res = []
    for k in range(1, 4):
        x, info = oracle.cg_ir(b, tol=0.0, max_outer=k, inner="f32", tol_in=1e-4, maxit_in=2000)
        res.append(info["relres_true"])
    assert res[0] <= 2e-4 and res[1] <= 2e-4 * res[0] * 10 and res[2] <= 1e-10
