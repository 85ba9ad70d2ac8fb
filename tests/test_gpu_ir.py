"""GPU mixed-precision solves (FP64 iterative refinement around a binary32 or
bf16-p/r inner classic CG) against the FP64 oracle.

Bar: the FP64 true residual reaches tol = 1e-10 and the solution is within
kappa * tol of a tightly converged FP64 oracle solution; refinement needs more
than one outer step (a binary32 inner solve alone cannot reach 1e-10)."""
import numpy as np
import pytest
import torch

import lap5_inputs as gen
import oracle
import paper_1803_03797_gb300 as lap5cg
from tests.helpers import rel_err

pytestmark = pytest.mark.gpu

SHAPES = [(1, 1), (3, 5), (64, 64), (100, 100), (130, 67), (255, 257)]


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda")


def _rel(a, b):
    return rel_err(a, b)  # norm-wise and element-wise


@pytest.mark.parametrize("precision", ["ir_f32", "ir_bf16pr"])
@pytest.mark.parametrize("nx,ny", SHAPES)
def test_ir_reaches_fp64_accuracy(precision, nx, ny):
    tol = 1e-10
    b = gen.uniform_rhs(nx, ny, seed=nx * 31 + ny, ld=gen.pitch(nx, 32))
    x, info = lap5cg.cg_solve(_dev(b), tol=tol, maxit=10 ** 6, precision=precision, nx=nx)
    rec = lap5cg.decode_info(info)[0]
    assert rec["status"] == lap5cg.OK, rec
    assert rec["relres_true"] <= tol
    xo, io = oracle.cg_classic(b, tol=1e-13, maxit=10 ** 6, nx=nx)
    kappa = gen.condition_number(nx, ny)
    assert _rel(x.cpu().numpy()[:, :nx], xo[:, :nx]) <= max(kappa * 2 * tol, 1e-13)
    if nx * ny > 16:
        assert rec["outer_iters"] >= 2
    # the oracle's refinement takes the same refinement steps and, within the
    # rounding of the inner dot products (binary32 Dot2 / bf16 storage summed in
    # another order), the same inner iterations: measured on a GB300, outer
    # steps equal on every shape here, inner totals within 1 (binary32) and
    # 3.5 % (bf16 p, r)
    xi, ii = oracle.cg_ir(b, tol=tol, inner="f32" if precision == "ir_f32" else "bf16pr", nx=nx)
    assert ii["status"] == oracle.OK
    assert abs(rec["outer_iters"] - ii["outer_iters"]) <= 1, (rec, ii)
    slack = max(3, ii["iters"] // 100) if precision == "ir_f32" else max(5, ii["iters"] // 20)
    assert abs(rec["iters"] - ii["iters"]) <= slack, (rec, ii)


@pytest.mark.parametrize("precision", ["ir_f32", "ir_bf16pr"])
def test_ir_edge_cases(precision):
    n = 48
    z = np.zeros((n, n))
    x, info = lap5cg.cg_solve(_dev(z), x0=_dev(np.ones((n, n))), tol=1e-10, maxit=100, precision=precision)
    rec = lap5cg.decode_info(info)[0]
    assert rec["status"] == lap5cg.OK and not x.cpu().numpy().any()
    b = gen.uniform_rhs(n, n, seed=1)
    b[5, 5] = np.inf
    x, info = lap5cg.cg_solve(_dev(b), tol=1e-10, maxit=100, precision=precision)
    assert lap5cg.decode_info(info)[0]["status"] == lap5cg.ERR_NONFINITE
    b = gen.uniform_rhs(n, n, seed=1)
    x, info = lap5cg.cg_solve(_dev(b), tol=1e-10, maxit=10, precision=precision)
    rec = lap5cg.decode_info(info)[0]
    assert rec["status"] == lap5cg.NOT_CONVERGED and rec["iters"] == 10


@pytest.mark.parametrize("precision", ["ir_f32", "ir_bf16pr"])
@pytest.mark.parametrize("nx,ny", [(1, 40), (100, 90), (129, 64), (257, 70), (300, 77), (1030, 120)])
def test_ir_inner_lane_vec_8(precision, nx, ny):
    # inner passes with eight columns a lane (two 16-byte groups 128 columns
    # apart, ring kernel), outer binary64 passes with two: ragged strips
    tol = 1e-10
    b = gen.uniform_rhs(nx, ny, seed=nx * 17 + ny, ld=gen.pitch(nx, 32))
    recs, xs = {}, {}
    for lv in (4, 8):
        opts = lap5cg.default_opts(lane_vec=lv, ring_slots=4)
        x, info = lap5cg.cg_solve(_dev(b), tol=tol, maxit=10 ** 6, precision=precision, nx=nx, opts=opts)
        recs[lv] = lap5cg.decode_info(info)[0]
        xs[lv] = x.cpu().numpy()[:, :nx]
        assert recs[lv]["status"] == lap5cg.OK and recs[lv]["relres_true"] <= tol, (lv, recs[lv])
    xo, io = oracle.cg_classic(b, tol=1e-13, maxit=10 ** 6, nx=nx)
    kappa = gen.condition_number(nx, ny)
    assert _rel(xs[8], xo[:, :nx]) <= max(kappa * 2 * tol, 1e-13)
    assert abs(recs[8]["outer_iters"] - recs[4]["outer_iters"]) <= 1


def test_ir_lane_vec_8_rejected_forms():
    b = _dev(gen.uniform_rhs(64, 64, seed=2))
    for opts in (dict(lane_vec=8, ring_slots=-1), dict(lane_vec=8, store_z=1, ring_slots=4)):
        with pytest.raises(lap5cg.Lap5cgError):
            lap5cg.cg_solve(b, tol=1e-10, precision="ir_f32", opts=lap5cg.default_opts(**opts))


def test_ir_newcg_inner_is_unsupported():
    b = _dev(gen.uniform_rhs(16, 16, seed=1))
    with pytest.raises(lap5cg.Lap5cgError):
        lap5cg.cg_solve(b, tol=1e-10, precision="ir_f32", variant="newcg")


def test_ir_2048_time_to_solution_beats_fp64():
    # config: 2048 x 2048 (the gradient workload's grid), to 1e-10
    n = 2048
    b = _dev(gen.uniform_rhs(n, n, seed=5))
    times = {}
    for precision in ("f64", "ir_f32"):
        lap5cg.cg_solve(b, tol=1e-10, maxit=10 ** 6, precision=precision)  # warm-up
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        x, info = lap5cg.cg_solve(b, tol=1e-10, maxit=10 ** 6, precision=precision)
        e1.record()
        torch.cuda.synchronize()
        rec = lap5cg.decode_info(info)[0]
        assert rec["status"] == lap5cg.OK and rec["relres_true"] <= 1.5e-10, (precision, rec)
        times[precision] = e0.elapsed_time(e1)
    assert times["ir_f32"] < times["f64"], times


def test_ir_8192_full_size_reaches_1e10():
    # the 8192 x 8192 mixed-precision workload at full size: FP64 true residual
    # recomputed by the oracle's stencil on the returned solution
    n = 8192
    b_np = gen.uniform_rhs(n, n, seed=3)
    x, info = lap5cg.cg_solve(_dev(b_np), tol=1e-10, maxit=10 ** 7, precision="ir_f32")
    rec = lap5cg.decode_info(info)[0]
    assert rec["status"] == lap5cg.OK and rec["relres_true"] <= 1e-10, rec
    x_np = x.cpu().numpy()
    res = b_np - oracle.lap5_apply(x_np)
    assert np.linalg.norm(res) <= 1.05e-10 * np.linalg.norm(b_np)


@pytest.mark.parametrize("precision", ["ir_f32", "ir_bf16pr"])
@pytest.mark.parametrize("n", [1024, 2048])
def test_ir_config_size_against_oracle_reference(precision, n):
    # the manufactured right-hand side at kappa = 4.3e5 / 1.7e6: the FP64 true
    # residual reaches 1e-10 and the solution is element-wise within the bound
    # ||x - x*||_inf <= ||b - A x||_2 / lambda_min of the oracle's multigrid
    # PCG solution x* (true residual ~5e-13)
    tol = 1e-10
    b = gen.manufactured_rhs(n, n, seed=2)
    xr, ir = oracle.cg_pcg(b, tol=1e-13, maxit=200)
    assert ir["status"] == oracle.OK
    x, info = lap5cg.cg_solve(_dev(b), tol=tol, maxit=10 ** 7, precision=precision)
    rec = lap5cg.decode_info(info)[0]
    assert rec["status"] == lap5cg.OK, rec
    assert rec["relres_true"] <= tol
    x = x.cpu().numpy()
    lam_min = gen.mode_eigenvalue(n, n, 1, 1)
    bound = (rec["relres_true"] + ir["relres_true"]) * np.linalg.norm(b) / lam_min
    assert np.linalg.norm(x - xr) <= bound
    assert np.max(np.abs(x - xr)) <= bound
    print("\n[error vs oracle] %s %d^2: %d refinements, %d inner iterations, relres_true %.3g, "
          "max|x - x*|/max|x*| %.3g (bound %.3g)" % (precision, n, rec["outer_iters"], rec["iters"],
                                                     rec["relres_true"], np.max(np.abs(x - xr)) / np.max(np.abs(xr)),
                                                     bound / np.max(np.abs(xr))))


# ---------------------------------------------------------------------------
# The refinement's guard: a step that raised the FP64 residual is kept when it
# lowered the error's energy (the oracle's rule), and undone at the FP64 floor.
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("batched", [False, True])
def test_ir_keeps_energy_lowering_steps_like_the_oracle(batched):
    # truncated bf16 inner solves (5 iterations): every other step raises the
    # 2-norm residual but lowers the energy; the oracle keeps all 12 steps
    n = 64
    b = gen.uniform_rhs(n, n, seed=81)
    _, io = oracle.cg_ir(b, tol=0.0, max_outer=12, inner="bf16pr", tol_in=1e-2, maxit_in=5)
    assert io["outer_iters"] == 12 and io["status"] == oracle.NOT_CONVERGED
    opts = lap5cg.default_opts(tol_inner=1e-2, maxit_inner=5, max_outer=12)
    if batched:  # the team kernel of the batched solve runs the same refinement
        _, info = lap5cg.cg_solve_batched([_dev(b)], tol=0.0, maxit=10 ** 6, precision="ir_bf16pr", opts=opts)
    else:
        _, info = lap5cg.cg_solve(_dev(b), tol=0.0, maxit=10 ** 6, precision="ir_bf16pr", opts=opts)
    rec = lap5cg.decode_info(info)[0]
    assert rec["status"] == lap5cg.NOT_CONVERGED and rec["outer_iters"] == 12 and rec["iters"] == 60, rec
    assert 0.5 * io["relres_true"] <= rec["relres_true"] <= 2.0 * io["relres_true"], (rec, io)


def test_ir_guard_undoes_a_step_at_the_fp64_floor():
    # binary32 inner solves run 384 iterations each: by the fourth step the
    # FP64 residual is at rounding level and the correction is noise
    n = 64
    b = gen.uniform_rhs(n, n, seed=81)
    _, io = oracle.cg_ir(b, tol=0.0, max_outer=6, inner="f32", tol_in=0.0, maxit_in=384)
    assert io["outer_iters"] < 6 and io["status"] == oracle.NOT_CONVERGED
    opts = lap5cg.default_opts(tol_inner=1e-300, maxit_inner=384, max_outer=6)
    x, info = lap5cg.cg_solve(_dev(b), tol=0.0, maxit=10 ** 6, precision="ir_f32", opts=opts)
    rec = lap5cg.decode_info(info)[0]
    assert rec["status"] == lap5cg.NOT_CONVERGED and rec["outer_iters"] < 6, rec
    assert rec["relres_true"] <= 1e-14
    # the undone step leaves the iterate before it: recursive = true residual
    assert abs(rec["relres_true"] - rec["relres_recursive"]) <= 1e-3 * rec["relres_true"]
