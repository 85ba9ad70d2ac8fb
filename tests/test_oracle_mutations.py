"""Planted mistakes: each test compiles a copy of the oracle with one plausible
error (a flipped sign, a wrong index, a dropped term, a swapped operand) and
checks that the pins catch it.  The mistakes are planted in a temporary copy on
the CPU; the committed oracle is never modified."""

import os
import subprocess

import numpy as np
import pytest
import scipy.linalg as sla

import lap5_inputs as gen
import oracle
from tests.helpers import flat, kron_laplacian

SRC = os.path.join(os.path.dirname(oracle.__file__), "lap5_oracle.c")

MUTATIONS = {
    "stencil_sign_west": ("acc -= at64(x, nx, ny, ld, i - 1, j);", "acc += at64(x, nx, ny, ld, i - 1, j);"),
    "stencil_index_north": ("acc -= at64(x, nx, ny, ld, i, j + 1);", "acc -= at64(x, nx, ny, ld, i + 1, j + 1);"),
    "classic_beta_inverted": ("double beta = gnew / gamma;                      /* (r,r)/(r_old,r_old) */",
                              "double beta = gamma / gnew;                      /* (r,r)/(r_old,r_old) */"),
    "classic_alpha_transposed": ("double alpha = gamma / pz;", "double alpha = pz / gamma;"),
    "newcg_r_sign": ("axpy64(nx, ny, ld, r, -alpha, q);                 /* r = r - alpha q */",
                     "axpy64(nx, ny, ld, r, alpha, q);                 /* r = r - alpha q */"),
    "newcg_w_uses_q": ("axpy64(nx, ny, ld, w, -alpha, z);                 /* w = w - alpha z */",
                       "axpy64(nx, ny, ld, w, -alpha, q);                 /* w = w - alpha z */"),
    "newcg_z_drops_beta": ("xpby64(nx, ny, ld, nv, beta, z);                  /* z = n + beta z */",
                           "xpby64(nx, ny, ld, nv, 0.0, z);                  /* z = n + beta z */"),
    "newcg_alpha_sign": ("double denom = delta / gamma - beta / alpha;    /* de-garbled alpha update */",
                         "double denom = delta / gamma + beta / alpha;    /* de-garbled alpha update */"),
    "newcg_stable_cross_term_sign": ("double pap = (delta + (2.0 * beta) * eps) + (beta * beta) * mu;",
                                     "double pap = (delta - (2.0 * beta) * eps) + (beta * beta) * mu;"),
    "newcg_stable_mu_dropped": ("double pap = (delta + (2.0 * beta) * eps) + (beta * beta) * mu;",
                                "double pap = (delta + (2.0 * beta) * eps);"),
}

# mistakes in the mixed-precision path, caught by the pins of tests/test_oracle_ir.py
IR_MUTATIONS = {
    "inner_beta_inverted": ("float bt = (float)(num / g);", "float bt = (float)(g / num);"),
    "inner_pr_beta_sign": ("double num = bf ? gn - dot2_pair(nx, ny, ld, r, rp) : gn;",
                           "double num = bf ? gn + dot2_pair(nx, ny, ld, r, rp) : gn;"),
    "inner_r_sign": ("r[t] = stor(r[t] - a * z[t], bf);", "r[t] = stor(r[t] + a * z[t], bf);"),
    "inner_p_not_rounded_to_bf16": ("p[t] = stor(r[t] + bt * p[t], bf);", "p[t] = r[t] + bt * p[t];"),
    "ir_update_sign": ("x[(size_t)j * ld + i] = x[(size_t)j * ld + i] + (double)d[(size_t)j * ld + i];",
                       "x[(size_t)j * ld + i] = x[(size_t)j * ld + i] - (double)d[(size_t)j * ld + i];"),
    "ir_guard_dropped": ("if (outer > 0 && !ora_ir_keep_step(", "if (0 && !ora_ir_keep_step("),
    "ir_keep_half_sign": ("return dro > 0.0 && drn >= -0.5 * dro;", "return dro > 0.0 && drn >= 0.5 * dro;"),
    "ir_keep_energy_ignored": ("return dro > 0.0 && drn >= -0.5 * dro;", "return 0;"),
    "ir_keep_claim_unchecked": ("return dro > 0.0 && drn >= -0.5 * dro;", "return drn >= -0.5 * dro;"),
}
MUTATIONS.update(IR_MUTATIONS)


@pytest.fixture(scope="module")
def mutant_dir(tmp_path_factory):
    return tmp_path_factory.mktemp("mutants")


def _load_mutant(name, mutant_dir):
    src = open(SRC).read()
    old, new = MUTATIONS[name]
    assert src.count(old) == 1, name
    path_c = os.path.join(mutant_dir, name + ".c")
    path_so = os.path.join(mutant_dir, name + ".so")
    with open(path_c, "w") as f:
        f.write(src.replace(old, new))
    subprocess.run(["gcc", "-O1", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared", "-o", path_so, path_c, "-lm"],
                   check=True)
    return path_so


class _Swap:
    def __init__(self, path):
        self.path = path

    def __enter__(self):
        self.saved = oracle._lib
        oracle._lib = None
        real_build = oracle._build.build
        oracle._build.build = lambda force=False: self.path
        try:
            oracle.lib()
        finally:
            oracle._build.build = real_build
        return self

    def __exit__(self, *exc):
        oracle._lib = self.saved
        return False


def _pins_pass():
    """A compact subset of the oracle pins; True iff all hold."""
    nx, ny = 9, 7
    xi = np.random.default_rng(0).integers(-50, 51, size=(ny, nx)).astype(np.float64)
    if not np.array_equal(flat(oracle.lap5_apply(xi), nx), kron_laplacian(nx, ny) @ flat(xi, nx)):
        return False
    A = kron_laplacian(nx, ny).toarray()
    b = gen.uniform_rhs(nx, ny, seed=3)
    x_ref = sla.cho_solve(sla.cho_factor(A), flat(b, nx))
    for variant in ("classic", "newcg"):
        x, info = oracle.cg_solve(b, variant=variant, tol=1e-12, maxit=400)
        if info["status"] != oracle.OK:
            return False
        if np.linalg.norm(flat(x, nx) - x_ref) > 1e-9 * np.linalg.norm(x_ref):
            return False
    for stable in (False, True):  # NewCG with its own and with the stabilised alpha
        x, info = oracle.cg_newcg(b, tol=1e-12, maxit=400, stable=stable)
        if info["status"] != oracle.OK or np.linalg.norm(flat(x, nx) - x_ref) > 1e-9 * np.linalg.norm(x_ref):
            return False
    n, K = 24, 12
    bb = gen.uniform_rhs(n, n, seed=5)
    tc = oracle.Trace(n, n, K + 1, K)
    tn = oracle.Trace(n, n, K + 1, K, newcg=True)
    oracle.cg_classic(bb, tol=0.0, maxit=K, trace=tc)
    oracle.cg_newcg(bb, tol=0.0, maxit=K, trace=tn)
    if not np.all(np.isfinite(tn.x[K])) or np.linalg.norm(tc.x[K] - tn.x[K]) > 1e-10 * np.linalg.norm(tc.x[K]):
        return False
    ts = oracle.Trace(n, n, K + 1, K, newcg=True)
    oracle.cg_newcg(bb, tol=0.0, maxit=K, trace=ts, stable=True)
    if not np.all(np.isfinite(ts.x[K])) or np.linalg.norm(tc.x[K] - ts.x[K]) > 1e-10 * np.linalg.norm(tc.x[K]):
        return False
    A2 = kron_laplacian(n, n)
    for k in range(K):
        w, r, z, q = (tn.w[k].reshape(-1), tn.r[k].reshape(-1), tn.z[k].reshape(-1), tn.q[k].reshape(-1))
        if np.linalg.norm(w - A2 @ r) > 1e-10 * np.linalg.norm(A2 @ r) or \
                np.linalg.norm(z - A2 @ q) > 1e-10 * np.linalg.norm(A2 @ q):
            return False
    return True


def _ir_pins_pass():
    """The mixed-precision pins (tests/test_oracle_ir.py); True iff all hold."""
    from tests import test_oracle_ir as t
    checks = [lambda: t.test_inner_one_step_on_sine_mode(3, 5),
              lambda: t.test_inner_m_modes_terminate_in_m_steps(0, 3),
              lambda: t.test_inner_f32_tracks_fp64_algorithm1(25),
              lambda: t.test_inner_matches_restatement_bit_for_bit("bf16pr"),
              lambda: t.test_inner_matches_restatement_bit_for_bit("f32"),
              lambda: t.test_refinement_equals_its_composition(40, "f32", 1e-4, 500, 3, False, False),
              lambda: t.test_refinement_equals_its_composition(64, "bf16pr", 1e-2, 5, 12, False, True),
              lambda: t.test_refinement_equals_its_composition(64, "f32", 0.0, 384, 6, True, False),
              t.test_keep_rule_follows_the_energy_definition]
    for check in checks:
        try:
            check()
        except (AssertionError, ValueError, FloatingPointError):
            return False
    return True


def test_unmutated_oracle_passes_pins():
    assert _pins_pass()
    assert _ir_pins_pass()


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_planted_mistake_is_caught(name, mutant_dir):
    path = _load_mutant(name, mutant_dir)
    with _Swap(path):
        caught = not (_ir_pins_pass() if name in IR_MUTATIONS else _pins_pass())
    assert caught, "pins did not catch the planted mistake " + name

