"""GPU parity of cg_solve (Algorithm 1 and Algorithm 2, binary64 and binary32)
against the oracle on the same seeded inputs.

Tolerances.  The GPU and the oracle take the same arithmetic steps but sum dot
products in different orders and the GPU fuses multiply-adds, so iterates
drift apart by rounding only: at a fixed iteration count k the binary64
solutions agree to ~1e-13 relative (asserted: 1e-10); converged solves agree in
iteration count within +-2 and in solution within kappa * tol.
"""
import math

import numpy as np
import pytest
import torch

import lap5_inputs as gen
import oracle
import paper_1803_03797_gb300 as lap5cg
from tests.helpers import rel_err

pytestmark = pytest.mark.gpu

VARIANTS = ["classic", "newcg"]


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda")


def _solve(b, **kw):
    x, info = lap5cg.cg_solve(_dev(b), **kw)
    return x.cpu().numpy(), lap5cg.decode_info(info)


def _rel(a, b):
    return rel_err(a, b)  # norm-wise and element-wise


SHAPES = [(1, 1), (1, 7), (7, 1), (2, 2), (3, 5), (16, 16), (33, 70), (100, 100), (130, 67), (255, 257)]


@pytest.mark.parametrize("resident", [0, -1])
@pytest.mark.parametrize("variant", VARIANTS)
@pytest.mark.parametrize("nx,ny", SHAPES)
def test_f64_converged_parity(variant, nx, ny, resident):
    # resident 0: small grids are solved inside one cluster's shared memory;
    # -1: the streaming kernels
    b = gen.uniform_rhs(nx, ny, seed=nx * 1000 + ny, ld=gen.pitch(nx, 8))
    tol = 1e-10
    x, info = _solve(b, tol=tol, maxit=20000, variant=variant, nx=nx, opts=lap5cg.default_opts(resident=resident))
    xo, io = oracle.cg_solve(b, variant=variant, tol=tol, maxit=20000, nx=nx)
    rec = info[0]
    assert rec["status"] == lap5cg.OK, rec
    assert abs(rec["iters"] - io["iters"]) <= 2, (rec, io)
    if variant == "classic":
        assert rec["relres_true"] <= 2 * tol
    else:
        # pipelined CG stops on its recursive residual; its true residual lags
        # behind (the oracle shows the same gap, e.g. 9.5e-10 at 255 x 257)
        assert rec["relres_true"] <= 3 * max(io["relres_true"], tol)
    kappa = gen.condition_number(nx, ny)
    assert _rel(x[:, :nx], xo[:, :nx]) <= max(kappa * max(tol, io["relres_true"]), 1e-12)


@pytest.mark.parametrize("resident", [0, -1])
@pytest.mark.parametrize("variant", VARIANTS)
@pytest.mark.parametrize("nx,ny,k", [(100, 100, 1), (100, 100, 7), (100, 100, 40), (257, 130, 25), (65, 64, 30)])
def test_f64_fixed_iteration_trajectory(variant, nx, ny, k, resident):
    b = gen.uniform_rhs(nx, ny, seed=k + nx, ld=gen.pitch(nx, 8))
    x, info = _solve(b, tol=0.0, maxit=k, variant=variant, nx=nx, opts=lap5cg.default_opts(resident=resident))
    xo, io = oracle.cg_solve(b, variant=variant, tol=0.0, maxit=k, nx=nx)
    assert info[0]["iters"] == io["iters"] == k
    assert info[0]["status"] == lap5cg.NOT_CONVERGED
    assert _rel(x[:, :nx], xo[:, :nx]) <= 1e-10
    assert abs(info[0]["relres_recursive"] - io["relres_recursive"]) <= 1e-9 * io["relres_recursive"]


@pytest.mark.parametrize("resident", [0, -1])
@pytest.mark.parametrize("variant", VARIANTS)
def test_residual_history_matches_oracle(variant, resident):
    n, K = 100, 120
    b = gen.uniform_rhs(n, n, seed=1)
    hist = torch.full((K + 1,), float("nan"), dtype=torch.float64, device="cuda")
    opts = lap5cg.default_opts(history=hist.data_ptr(), resident=resident)
    lap5cg.cg_solve(_dev(b), tol=0.0, maxit=K, variant=variant, opts=opts)
    tr = oracle.Trace(n, n, 1, K, newcg=(variant == "newcg"))
    oracle.cg_solve(b, variant=variant, tol=0.0, maxit=K, trace=tr)
    h = hist.cpu().numpy()
    np.testing.assert_allclose(h, tr.relres, rtol=1e-7)


@pytest.mark.parametrize("store_z", [0, 1])
def test_classic_store_z_and_recompute_agree(store_z):
    n = 200
    b = gen.uniform_rhs(n, n, seed=5)
    x, info = _solve(b, tol=0.0, maxit=60, variant="classic", opts=lap5cg.default_opts(store_z=store_z, resident=-1))
    xo, _ = oracle.cg_classic(b, tol=0.0, maxit=60)
    assert _rel(x, xo) <= 1e-10


@pytest.mark.parametrize("ctas,warps,min_rows", [(1, 4, 1), (3, 8, 5), (0, 16, 64), (7, 2, 3)])
def test_launch_geometries_agree(ctas, warps, min_rows):
    nx, ny = 300, 170
    b = gen.uniform_rhs(nx, ny, seed=9, ld=gen.pitch(nx, 8))
    opts = lap5cg.default_opts(ctas=ctas, warps_per_cta=warps, min_rows=min_rows, resident=-1)
    for variant in VARIANTS:
        x, info = _solve(b, tol=0.0, maxit=30, variant=variant, nx=nx, opts=opts)
        xo, _ = oracle.cg_solve(b, variant=variant, tol=0.0, maxit=30, nx=nx)
        assert _rel(x[:, :nx], xo[:, :nx]) <= 1e-10


@pytest.mark.parametrize("variant", VARIANTS)
def test_edge_cases(variant):
    n = 40
    b = np.zeros((n, n))
    x0 = np.ones((n, n))
    x, info = lap5cg.cg_solve(_dev(b), x0=_dev(x0), tol=1e-8, maxit=10, variant=variant)
    rec = lap5cg.decode_info(info)[0]
    assert rec["status"] == lap5cg.OK and rec["iters"] == 0 and not x.cpu().numpy().any()
    b = gen.uniform_rhs(n, n, seed=2)
    x, info = _solve(b, tol=1e-8, maxit=0, variant=variant)
    assert info[0]["status"] == lap5cg.NOT_CONVERGED and info[0]["iters"] == 0 and not x.any()
    x, info = _solve(b, tol=-1.0, maxit=13, variant=variant)
    assert info[0]["status"] == lap5cg.NOT_CONVERGED and info[0]["iters"] == 13
    bn = b.copy()
    bn[3, 4] = np.nan
    x, info = _solve(bn, tol=1e-8, maxit=10, variant=variant)
    assert info[0]["status"] == lap5cg.ERR_NONFINITE and not x.any()
    # exact one-step termination on the manufactured (1,1) mode
    lam = gen.mode_eigenvalue(n, n, 1, 1)
    u = gen.sine_mode(n, n, 1, 1)
    x, info = _solve(lam * u, tol=1e-12, maxit=5, variant=variant)
    assert info[0]["iters"] == 1 and np.abs(x - u).max() <= 1e-13


@pytest.mark.parametrize("variant", VARIANTS)
def test_initial_guess_resume(variant):
    n = 96
    b = gen.uniform_rhs(n, n, seed=4)
    x1, _ = _solve(b, tol=0.0, maxit=50, variant=variant)
    x, info = lap5cg.cg_solve(_dev(b), x0=_dev(x1), tol=1e-10, maxit=5000, variant=variant)
    xo, io = oracle.cg_solve(b, variant=variant, x0=x1, tol=1e-10, maxit=5000)
    rec = lap5cg.decode_info(info)[0]
    assert rec["status"] == lap5cg.OK and abs(rec["iters"] - io["iters"]) <= 2
    assert rec["relres_true"] <= 2e-10


@pytest.mark.parametrize("variant", VARIANTS)
@pytest.mark.parametrize("nx,ny,ld", [(101, 37, 101), (63, 64, 63), (5, 3, 5)])
def test_unaligned_pitch_is_staged(variant, nx, ny, ld):
    b = gen.uniform_rhs(nx, ny, seed=3, ld=ld)
    x, info = _solve(b, tol=0.0, maxit=25, variant=variant, nx=nx)
    xo, _ = oracle.cg_solve(b, variant=variant, tol=0.0, maxit=25, nx=nx)
    assert _rel(x[:, :nx], xo[:, :nx]) <= 1e-10


@pytest.mark.parametrize("variant", VARIANTS)
def test_multiple_rhs(variant):
    n, k = 64, 3
    bs = np.stack([gen.uniform_rhs(n, n, seed=s) for s in range(k)])
    x, info = lap5cg.cg_solve(_dev(bs), tol=1e-10, maxit=5000, variant=variant)
    recs = lap5cg.decode_info(info)
    x = x.cpu().numpy()
    for s in range(k):
        xo, io = oracle.cg_solve(bs[s], variant=variant, tol=1e-10, maxit=5000)
        assert recs[s]["status"] == lap5cg.OK and abs(recs[s]["iters"] - io["iters"]) <= 2
        assert _rel(x[s], xo) <= gen.condition_number(n, n) * 1e-10


def test_newcg_residual_replacement():
    n = 128
    b = gen.uniform_rhs(n, n, seed=21)
    opts = lap5cg.default_opts(rr_period=25)
    x, info = _solve(b, tol=0.0, maxit=80, variant="newcg", opts=opts)
    xo, io = oracle.cg_newcg(b, tol=0.0, maxit=80, rr_period=25)
    assert _rel(x, xo) <= 1e-10
    x, info = _solve(b, tol=1e-12, maxit=5000, variant="newcg", opts=opts)
    assert info[0]["status"] == lap5cg.OK and info[0]["relres_true"] <= 2e-12


@pytest.mark.parametrize("nx,ny", [(1, 1), (3, 5), (100, 100), (129, 131)])
def test_f32_classic(nx, ny):
    b = gen.uniform_rhs(nx, ny, seed=nx + ny, ld=gen.pitch(nx, 4)).astype(np.float32)
    tol = 1e-5
    x, info = _solve(b, tol=tol, maxit=20000, variant="classic", precision="f32", nx=nx)
    rec = info[0]
    assert rec["status"] == lap5cg.OK, rec
    xo, io = oracle.cg_solve(b.astype(np.float64), variant="classic", tol=1e-13, maxit=20000, nx=nx)
    kappa = gen.condition_number(nx, ny)
    err = _rel(x[:, :nx].astype(np.float64), xo[:, :nx])
    # binary32 storage adds ~kappa * u32 of error on top of the tolerance
    assert err <= kappa * (2 * tol + 4 * 2.0 ** -24)
    assert rec["relres_true"] <= 2 * tol + 50 * 2.0 ** -24 * math.sqrt(nx * ny)


@pytest.mark.parametrize("variant", VARIANTS)
@pytest.mark.parametrize("nx,ny,k", [(100, 100, 30), (129, 131, 40), (3, 5, 4)])
def test_f32_fixed_iterations_track_fp64_oracle(variant, nx, ny, k):
    b = gen.uniform_rhs(nx, ny, seed=7 * nx + ny, ld=gen.pitch(nx, 4)).astype(np.float32)
    x, info = _solve(b, tol=0.0, maxit=k, variant=variant, precision="f32", nx=nx)
    xo, io = oracle.cg_solve(b.astype(np.float64), variant=variant, tol=0.0, maxit=k, nx=nx)
    assert info[0]["iters"] == min(k, io["iters"])
    # binary32 rounding drift over k steps; the pipelined recurrences amplify
    # it (measured 1.2e-4 / 2.4e-4 for NewCG here, 1e-6-level for classic)
    assert _rel(x[:, :nx].astype(np.float64), xo[:, :nx]) <= (1e-4 if variant == "classic" else 1e-3)


@pytest.mark.parametrize("nx,ny", [(1, 9), (5, 40), (127, 33), (128, 30), (129, 41), (255, 64), (256, 64),
                                   (257, 70), (300, 77), (513, 100), (1100, 64)])
def test_f32_lane_vec_8_tracks_oracle_and_lane_vec_4(nx, ny):
    # eight columns a lane (two 16-byte groups 128 columns apart): ragged
    # strips where the second group is partly or wholly outside the grid
    b = gen.uniform_rhs(nx, ny, seed=5 * nx + ny, ld=gen.pitch(nx, 4)).astype(np.float32)
    k = 25
    xs = {}
    for lv in (4, 8):
        opts = lap5cg.default_opts(lane_vec=lv, ring_slots=4)
        x, info = _solve(b, tol=0.0, maxit=k, variant="classic", precision="f32", nx=nx, opts=opts)
        xs[lv] = x[:, :nx].astype(np.float64)
        assert info[0]["iters"] <= k and info[0]["status"] in (lap5cg.OK, lap5cg.NOT_CONVERGED)
    xo, io = oracle.cg_classic(b.astype(np.float64), tol=0.0, maxit=k, nx=nx)
    assert _rel(xs[8], xo[:, :nx]) <= 1e-4
    # the two layouts differ only in the order of dot-product partial sums
    assert _rel(xs[8], xs[4]) <= 1e-4
    assert np.isfinite(xs[8]).all()


def test_f32_lane_vec_8_converged_and_rejected_forms():
    nx, ny = 1030, 300
    b = gen.uniform_rhs(nx, ny, seed=91, ld=gen.pitch(nx, 4)).astype(np.float32)
    tol = 1e-5
    # explicit ring: at this size the automatic choice would take the register
    # march (units shorter than 8 rows), which has no eight-column form
    x, info = _solve(b, tol=tol, maxit=20000, variant="classic", precision="f32", nx=nx,
                     opts=lap5cg.default_opts(lane_vec=8, ring_slots=4))
    rec = info[0]
    assert rec["status"] == lap5cg.OK, rec
    xo, io = oracle.cg_solve(b.astype(np.float64), variant="classic", tol=1e-13, maxit=20000, nx=nx)
    kappa = gen.condition_number(nx, ny)
    assert _rel(x[:, :nx].astype(np.float64), xo[:, :nx]) <= kappa * (2 * tol + 4 * 2.0 ** -24)
    # eight columns a lane exist for the ring kernel of classic CG only
    for kw in (dict(variant="newcg"), dict(variant="classic", opts_extra=dict(ring_slots=-1))):
        extra = kw.pop("opts_extra", {})
        with pytest.raises(RuntimeError):
            _solve(b, tol=tol, maxit=10, precision="f32", nx=nx, opts=lap5cg.default_opts(lane_vec=8, **extra), **kw)
    with pytest.raises(RuntimeError):
        _solve(b, tol=tol, maxit=10, precision="f32", nx=nx, opts=lap5cg.default_opts(lane_vec=6))


@pytest.mark.parametrize("nx,ny", [(1, 9), (3, 40), (127, 33), (128, 30), (129, 41), (255, 64), (300, 77),
                                   (513, 100)])
@pytest.mark.parametrize("store_z", [0, 1])
def test_f64_lane_vec_4_tracks_oracle_and_lane_vec_2(nx, ny, store_z):
    # four binary64 columns a lane (32 bytes, ring kernel of classic CG):
    # ragged strips of 128 columns, both z forms
    b = gen.uniform_rhs(nx, ny, seed=3 * nx + ny, ld=gen.pitch(nx, 8, 32))
    k = 25
    xs = {}
    for lv in (2, 4):
        opts = lap5cg.default_opts(lane_vec=lv, ring_slots=4, store_z=store_z)
        x, info = _solve(b, tol=0.0, maxit=k, variant="classic", nx=nx, opts=opts)
        xs[lv] = x[:, :nx]
        assert info[0]["iters"] <= k and info[0]["status"] in (lap5cg.OK, lap5cg.NOT_CONVERGED)
    xo, io = oracle.cg_classic(b, tol=0.0, maxit=k, nx=nx)
    assert _rel(xs[4], xo[:, :nx]) <= 1e-10
    assert _rel(xs[4], xs[2]) <= 1e-10


def test_f64_lane_vec_rejected_forms():
    nx, ny = 200, 50
    b4 = gen.uniform_rhs(nx, ny, seed=8, ld=gen.pitch(nx, 8, 32))
    b2 = gen.uniform_rhs(nx, ny, seed=8, ld=202)  # a pitch of two (not four) columns
    # (resident=-1: the streaming kernels; a grid this small would otherwise be
    # solved in one cluster's shared memory, which has no lane-vector choice)
    # the automatic choice falls back to two columns where four are not available
    for b, opts in ((b2, {}), (b4, dict(ring_slots=-1)), (b4, dict(reproducible=1))):
        x, info = _solve(b, tol=1e-10, maxit=2000, nx=nx, opts=lap5cg.default_opts(resident=-1, **opts))
        assert info[0]["status"] == lap5cg.OK
    for b, variant, opts in ((b2, "classic", dict(lane_vec=4)), (b4, "newcg", dict(lane_vec=4)),
                             (b4, "classic", dict(lane_vec=4, ring_slots=-1)),
                             (b4, "classic", dict(lane_vec=4, reproducible=1)), (b4, "classic", dict(lane_vec=8))):
        with pytest.raises(RuntimeError):
            _solve(b, tol=1e-10, maxit=10, variant=variant, nx=nx, opts=lap5cg.default_opts(resident=-1, **opts))
    with pytest.raises(RuntimeError):  # binary32 passes have no two-column form
        _solve(b4.astype(np.float32), tol=1e-5, maxit=10, precision="f32", nx=nx,
               opts=lap5cg.default_opts(lane_vec=2, resident=-1))


def test_f32_full_size_8192_fused_launch_tracks_oracle():
    # the 8192 x 8192 binary32 fused-iteration workload in its timed launch
    # configuration (automatic lane vector: 8), fixed iterations, against the
    # binary64 oracle
    n, k = 8192, 6
    b = gen.uniform_rhs(n, n, seed=3).astype(np.float32)
    x, info = _solve(b, tol=0.0, maxit=k, variant="classic", precision="f32",
                     opts=lap5cg.default_opts(true_residual=0))
    assert info[0]["iters"] == k
    xo, io = oracle.cg_classic(b.astype(np.float64), tol=0.0, maxit=k)
    assert _rel(x.astype(np.float64), xo) <= 1e-5
    assert abs(info[0]["relres_recursive"] - io["relres_recursive"]) <= 1e-4 * io["relres_recursive"]


def test_f32_newcg_limited_accuracy_reports_breakdown():
    # Binary32 pipelined CG loses the accuracy of its w/q/z recurrences: an
    # independent numpy binary32 restatement of Algorithm 2 breaks down at
    # iteration ~220 on this grid too.  The kernel must stop with a clean
    # status (no hang) either way.
    b = gen.uniform_rhs(100, 100, seed=200).astype(np.float32)
    x, info = _solve(b, tol=1e-7, maxit=20000, variant="newcg", precision="f32")
    rec = info[0]
    assert rec["status"] in (lap5cg.OK, lap5cg.ERR_BREAKDOWN)
    assert 0 < rec["iters"] < 20000
    assert np.isfinite(x).all()


@pytest.mark.parametrize("variant", VARIANTS)
def test_full_size_4096_trajectory(variant):
    # the benchmark's workload exactly: 4096 x 4096 binary64, the manufactured
    # right-hand side, 500 iterations, the benchmark's launch configuration;
    # element-wise against the oracle's iterate at the same count (the oracle
    # needs about a minute a variant)
    # Bound: the trajectory's sensitivity to the order of dot-product sums.
    # The oracle's own NewCG moves by 1.45e-9 here when only its summation
    # order changes (sequential against per-thread partial sums); the
    # pipelined recurrences amplify rounding more than Algorithm 1's.  A wrong
    # halo, index or coefficient shows at 1e-4 and above.
    n, k = 4096, 500
    bound = {"classic": 1e-10, "newcg": 1e-8}[variant]
    b = gen.manufactured_rhs(n, n, seed=2)
    x, info = _solve(b, tol=0.0, maxit=k, variant=variant)
    xo, io = oracle.cg_solve(b, variant=variant, tol=0.0, maxit=k)
    assert info[0]["iters"] == io["iters"] == k
    assert _rel(x, xo) <= bound
    assert np.max(np.abs(x - xo)) <= bound * np.max(np.abs(xo))
    assert abs(info[0]["relres_recursive"] - io["relres_recursive"]) <= 1e-8 * io["relres_recursive"]
    assert abs(info[0]["relres_true"] - io["relres_true"]) <= 1e-8 * io["relres_true"]
    print("\n[trajectory 4096^2 k=500] %s: rel diff vs oracle %.3g" % (variant, _rel(x, xo)))


_REF = {}


def _reference_4096():
    """x* for the 4096^2 manufactured problem: the oracle's multigrid PCG to a
    recursive residual of 1e-13 (true residual ~5e-13), about 25 s on the host."""
    if "x" not in _REF:
        b = gen.manufactured_rhs(4096, 4096, seed=2)
        x, info = oracle.cg_pcg(b, tol=1e-13, maxit=200)
        assert info["status"] == oracle.OK
        _REF.update(b=b, x=x, info=info)
    return _REF["b"], _REF["x"], _REF["info"]


@pytest.mark.parametrize("name,variant,precision,rr", [
    ("f64_classic", "classic", "f64", 0), ("f64_newcg_rr100", "newcg", "f64", 100),
    ("f64_newcg_stable_rr100", "newcg", "f64", -100), ("ir_f32", "classic", "ir_f32", 0),
    ("ir_bf16pr", "classic", "ir_bf16pr", 0), ("pcg_mg_f32", "classic", "mg_f32", 0),
    ("pcg_mg_f64", "classic", "mg_f64", 0), ("pipelined_pcg_mg_f64", "newcg", "mg_f64", 0)])
def test_full_size_4096_converged_error_vs_oracle(name, variant, precision, rr):
    # Every solver of the time-to-1e-10 comparison at the benchmark size
    # (kappa = 6.8e6), element-wise against an oracle solution 200x tighter.
    # Bound: ||x - x*||_inf <= ||x - x*||_2 <= ||b - A x||_2 / lambda_min, with
    # the true residual the solve reports (plus the reference's own).
    b, xr, ir = _reference_4096()
    n, tol = 4096, 1e-10
    x, info = _solve(b, tol=tol, maxit=10 ** 7, variant=variant, precision=precision,
                     opts=lap5cg.default_opts(rr_period=abs(rr), stabilized=int(rr < 0)))
    rec = info[0]
    assert rec["status"] == lap5cg.OK, rec
    assert rec["relres_true"] <= 1.5 * tol, rec
    lam_min = gen.mode_eigenvalue(n, n, 1, 1)
    res = (rec["relres_true"] + ir["relres_true"]) * np.linalg.norm(b)
    err_max = float(np.max(np.abs(x - xr)))
    err_norm = float(np.linalg.norm(x - xr))
    assert err_norm <= res / lam_min
    assert err_max <= res / lam_min
    print("\n[error vs oracle] %s: iters %d, relres_true %.3g, max|x - x*|/max|x*| %.3g, "
          "||x - x*||/||x*|| %.3g, bound %.3g" % (name, rec["iters"], rec["relres_true"],
                                                 err_max / np.max(np.abs(xr)), err_norm / np.linalg.norm(xr),
                                                 res / lam_min / np.max(np.abs(xr))))


def test_full_size_4096_500_iterations_properties():
    n = 4096
    b = gen.manufactured_rhs(n, n, seed=2)
    recs = {}
    for variant in VARIANTS:
        x, info = _solve(b, tol=0.0, maxit=500, variant=variant)
        rec = info[0]
        assert rec["iters"] == 500 and rec["status"] == lap5cg.NOT_CONVERGED
        # the recurrence residual still tracks the true residual after 500 steps
        assert abs(rec["relres_true"] - rec["relres_recursive"]) <= 1e-6 * rec["relres_true"] + 1e-13
        assert rec["relres_true"] < 0.05
        recs[variant] = rec
    # both variants follow the same Krylov sequence
    assert abs(recs["classic"]["relres_true"] - recs["newcg"]["relres_true"]) <= 1e-6 * recs["classic"]["relres_true"]


@pytest.mark.parametrize("ring_slots", [-1, 3, 8])
def test_ring_and_register_paths_agree(ring_slots):
    # rows staged through the shared-memory ring (3 or 8 slots) or loaded into
    # registers (-1): same arithmetic, same results against the oracle
    nx, ny = 301, 170
    b = gen.uniform_rhs(nx, ny, seed=77, ld=gen.pitch(nx, 32))
    for variant in VARIANTS:
        for store_z in (0, 1):
            if variant == "newcg" and store_z:
                continue
            opts = lap5cg.default_opts(ring_slots=ring_slots, store_z=store_z)
            x, info = _solve(b, tol=0.0, maxit=30, variant=variant, nx=nx, opts=opts)
            xo, _ = oracle.cg_solve(b, variant=variant, tol=0.0, maxit=30, nx=nx)
            assert info[0]["status"] == lap5cg.NOT_CONVERGED
            assert _rel(x[:, :nx], xo[:, :nx]) <= 1e-10
    bf = b.astype(np.float32)
    x, info = _solve(bf, tol=0.0, maxit=30, variant="classic", precision="f32", nx=nx,
                     opts=lap5cg.default_opts(ring_slots=ring_slots))
    xo, _ = oracle.cg_classic(bf.astype(np.float64), tol=0.0, maxit=30, nx=nx)
    assert _rel(x[:, :nx].astype(np.float64), xo[:, :nx]) <= 1e-4
    for precision in ("ir_f32", "ir_bf16pr"):
        x, info = _solve(b, tol=1e-10, maxit=10 ** 6, precision=precision, nx=nx,
                         opts=lap5cg.default_opts(ring_slots=ring_slots))
        assert info[0]["status"] == lap5cg.OK and info[0]["relres_true"] <= 1e-10


@pytest.mark.parametrize("variant", VARIANTS)
@pytest.mark.parametrize("nx,ny", [(1, 200000), (200000, 1), (3, 70001)])
def test_extreme_aspect_ratios(variant, nx, ny):
    # one-row / one-column grids: many strips or many row segments.  kappa is
    # about 3 here, so 20 steps stay well above rounding level
    b = gen.uniform_rhs(nx, ny, seed=nx + ny, ld=gen.pitch(nx, 8))
    x, info = _solve(b, tol=0.0, maxit=20, variant=variant, nx=nx)
    xo, io = oracle.cg_solve(b, variant=variant, tol=0.0, maxit=20, nx=nx)
    assert info[0]["iters"] == io["iters"]
    assert _rel(x[:, :nx], xo[:, :nx]) <= 1e-10


# ---------------------------------------------------------------------------
# NewCG with the stabilised alpha (alpha = gamma / (p, A p), (p, A p) from dot
# products of the current vectors) against the oracle's stabilised NewCG
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("precision", ["f64", "f32"])
@pytest.mark.parametrize("nx,ny,k", [(100, 100, 40), (257, 130, 25), (65, 64, 30), (3, 5, 4)])
def test_newcg_stable_trajectory(precision, nx, ny, k):
    dt = np.float64 if precision == "f64" else np.float32
    b = gen.uniform_rhs(nx, ny, seed=k + 3 * nx, ld=gen.pitch(nx, 8)).astype(dt)
    x, info = _solve(b, tol=0.0, maxit=k, variant="newcg", precision=precision, nx=nx,
                     opts=lap5cg.default_opts(stabilized=1))
    xo, io = oracle.cg_newcg(b.astype(np.float64), tol=0.0, maxit=k, nx=nx, stable=True)
    assert info[0]["iters"] == min(k, io["iters"])
    bound = 1e-10 if precision == "f64" else 1e-3  # binary32: rounding drift of the pipelined recurrences
    assert _rel(x[:, :nx].astype(np.float64), xo[:, :nx]) <= bound


@pytest.mark.parametrize("rr", [0, 25])
@pytest.mark.parametrize("nx,ny", [(100, 100), (255, 257), (33, 70)])
def test_newcg_stable_converged(nx, ny, rr):
    b = gen.uniform_rhs(nx, ny, seed=nx + 11 * ny, ld=gen.pitch(nx, 8))
    tol = 1e-10
    x, info = _solve(b, tol=tol, maxit=20000, variant="newcg", nx=nx,
                     opts=lap5cg.default_opts(stabilized=1, rr_period=rr))
    xo, io = oracle.cg_newcg(b, tol=tol, maxit=20000, nx=nx, rr_period=rr, stable=True)
    rec = info[0]
    assert rec["status"] == lap5cg.OK and io["status"] == oracle.OK, (rec, io)
    assert abs(rec["iters"] - io["iters"]) <= 2
    kappa = gen.condition_number(nx, ny)
    assert _rel(x[:, :nx], xo[:, :nx]) <= kappa * max(tol, io["relres_true"])
    assert rec["relres_true"] <= 3 * max(io["relres_true"], tol)


def test_newcg_stable_survives_where_algorithm2_breaks_down():
    # 128^2 to 1e-15 with replacement every 100: Algorithm 2's recurrence for
    # alpha breaks down near the attainable accuracy, the stabilised form does
    # not (the oracle shows the same, tests/test_oracle_cg.py)
    n = 128
    b = gen.manufactured_rhs(n, n, seed=2)
    _, info = _solve(b, tol=1e-15, maxit=2000, variant="newcg", opts=lap5cg.default_opts(rr_period=100, resident=-1))
    assert info[0]["status"] == lap5cg.ERR_BREAKDOWN
    x, info = _solve(b, tol=1e-15, maxit=2000, variant="newcg",
                     opts=lap5cg.default_opts(rr_period=100, stabilized=1))
    assert info[0]["status"] == lap5cg.NOT_CONVERGED and info[0]["iters"] == 2000
    assert info[0]["relres_true"] <= 1e-11


def test_newcg_stable_rejected_forms():
    b = gen.uniform_rhs(64, 64, seed=5)
    with pytest.raises(lap5cg.Lap5cgError) as e:
        _solve(b, tol=1e-10, maxit=10, variant="classic", opts=lap5cg.default_opts(stabilized=1))
    assert e.value.code == lap5cg.ERR_INVALID_ARG
    for kw in (dict(precision="ir_f32"), dict(precision="mg_f64"), dict(opts_extra=dict(reproducible=1))):
        extra = kw.pop("opts_extra", {})
        with pytest.raises(lap5cg.Lap5cgError) as e:
            _solve(b, tol=1e-10, maxit=10, variant="newcg", opts=lap5cg.default_opts(stabilized=1, **extra), **kw)
        assert e.value.code == lap5cg.ERR_UNSUPPORTED
    with pytest.raises(lap5cg.Lap5cgError) as e:
        lap5cg.cg_solve_batched([_dev(b)], tol=1e-10, variant="newcg", precision="f64",
                                opts=lap5cg.default_opts(stabilized=1))
    assert e.value.code == lap5cg.ERR_UNSUPPORTED
