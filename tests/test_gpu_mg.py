"""GPU multigrid-preconditioned CG (precision "mg_f64" / "mg_f32": binary64
PCG with a binary64 / binary32 V-cycle as M^-1) against the oracle's cg_pcg.

Tolerances.  With the V-cycle in binary64 the GPU and the oracle take the same
steps in the same association order; they differ in fused multiply-adds
(Jacobi sweeps, vector updates) and in the order of dot-product partial sums,
so fixed-iteration iterates agree to rounding level (asserted 1e-11 relative).
A binary32 V-cycle is a slightly different (rounded) preconditioner: converged
solves reach the same tolerance in about the same number of iterations."""
import numpy as np
import pytest
import torch

import lap5_inputs as gen
import oracle
import paper_1803_03797_gb300 as lap5cg
from tests.helpers import rel_err

pytestmark = pytest.mark.gpu


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda")


def _solve(b, nx, precision, tol, maxit, variant="classic", **opt):
    x, info = lap5cg.cg_solve(_dev(b), tol=tol, maxit=maxit, precision=precision, nx=nx, variant=variant,
                              opts=lap5cg.default_opts(**opt))
    return x.cpu().numpy()[:, :nx], lap5cg.decode_info(info)[0]


def _rel(a, b):
    return rel_err(a, b)  # norm-wise and element-wise


# (1, 1) .. (63, 63): the whole hierarchy on one CTA; (300, 200): levels 0 and 1
# grid-wide, the rest on one CTA; (1, 200), (200, 1): no coarse grid at all
SHAPES = [(1, 1), (2, 2), (3, 5), (15, 15), (16, 16), (63, 63), (100, 100), (130, 67), (300, 200), (255, 257),
          (1, 200), (200, 1), (513, 130), (1000, 9), (3, 8000)]
# (1000, 9): level 1 (499 x 4) is the coarsest and fits one CTA's shared
# memory; (3, 8000): level 1 (1 x 3999) has a pitch of 4, too large for shared
# memory, so its single-CTA kernel works in global memory


@pytest.mark.parametrize("nx,ny", SHAPES)
def test_fixed_iterations_track_oracle_f64_vcycle(nx, ny):
    b = gen.uniform_rhs(nx, ny, seed=nx * 3 + ny, ld=gen.pitch(nx, 8))
    for k in (1, 3, 6):
        x, rec = _solve(b, nx, "mg_f64", 0.0, k)
        xo, io = oracle.cg_pcg(b, tol=0.0, maxit=k, nx=nx)
        assert rec["iters"] == io["iters"], (k, rec, io)
        assert rec["status"] == io["status"], (k, rec, io)
        assert _rel(x, xo[:, :nx]) <= 1e-11, (k, _rel(x, xo[:, :nx]))


@pytest.mark.parametrize("precision", ["mg_f64", "mg_f32"])
@pytest.mark.parametrize("nx,ny", [(63, 63), (100, 100), (300, 200), (513, 130), (1, 200)])
def test_converged_solve_matches_oracle(precision, nx, ny):
    tol = 1e-10
    b = gen.uniform_rhs(nx, ny, seed=nx + 5 * ny, ld=gen.pitch(nx, 8))
    x, rec = _solve(b, nx, precision, tol, 500)
    xo, io = oracle.cg_pcg(b, tol=tol, maxit=500, nx=nx)
    assert rec["status"] == lap5cg.OK, rec
    assert rec["relres_true"] <= 1.5 * tol
    slack = 2 if precision == "mg_f64" else 4
    assert abs(rec["iters"] - io["iters"]) <= slack, (rec, io)
    xt, _ = oracle.cg_pcg(b, tol=1e-13, maxit=500, nx=nx)
    assert _rel(x, xt[:, :nx]) <= gen.condition_number(nx, ny) * 2 * tol


@pytest.mark.parametrize("opt", [dict(mg_nu=1), dict(mg_nu=3), dict(mg_levels=1), dict(mg_levels=2),
                                 dict(mg_coarse_sweeps=3), dict(warps_per_cta=4), dict(ctas=40)])
def test_options_track_oracle(opt):
    nx, ny = 300, 200
    b = gen.uniform_rhs(nx, ny, seed=17, ld=gen.pitch(nx, 8))
    k = 5
    x, rec = _solve(b, nx, "mg_f64", 0.0, k, **opt)
    ok = {"levels": opt.get("mg_levels", oracle.MG_LEVELS) or oracle.MG_LEVELS, "nu": opt.get("mg_nu", 2),
          "nu_coarse": opt.get("mg_coarse_sweeps", 8)}
    xo, io = oracle.cg_pcg(b, tol=0.0, maxit=k, nx=nx, **ok)
    assert rec["iters"] == io["iters"] == k
    assert _rel(x, xo[:, :nx]) <= 1e-11


def test_edge_cases_and_rejections():
    n = 48
    z = np.zeros((n, n))
    x, rec = _solve(z, n, "mg_f32", 1e-10, 100)
    assert rec["status"] == lap5cg.OK and rec["iters"] == 0 and not x.any()
    b = gen.uniform_rhs(n, n, seed=1)
    b[5, 5] = np.inf
    x, rec = _solve(b, n, "mg_f32", 1e-10, 100)
    assert rec["status"] == lap5cg.ERR_NONFINITE
    bd = _dev(gen.uniform_rhs(n, n, seed=1))
    with pytest.raises(lap5cg.Lap5cgError):
        lap5cg.cg_solve(bd, tol=1e-10, precision="mg_f32", opts=lap5cg.default_opts(mg_nu=-1))


@pytest.mark.parametrize("precision", ["mg_f32", "mg_f64"])
def test_full_size_4096_reaches_1e10(precision):
    # the 4096 x 4096 benchmark grid and right-hand side, to 1e-10; the true
    # residual recomputed by the oracle's stencil
    n = 4096
    b = gen.manufactured_rhs(n, n, seed=2)
    x, rec = _solve(b, n, precision, 1e-10, 200)
    assert rec["status"] == lap5cg.OK and rec["iters"] <= 30, rec
    res = b - oracle.lap5_apply(x)
    assert np.linalg.norm(res) <= 1.05e-10 * np.linalg.norm(b)


# ---------------------------------------------------------------------------
# Pipelined form (variant "newcg"): oracle.cg_ppcg
# ---------------------------------------------------------------------------
# Tiny grids are left out: the preconditioned solve reaches rounding level in a
# few steps, after which the recurrences (and where they break down) are
# rounding noise that fused multiply-adds change
@pytest.mark.parametrize("nx,ny", [(5, 40), (17, 33), (16, 16), (63, 63), (100, 100), (300, 200), (1, 200), (513, 130)])
def test_pipelined_fixed_iterations_track_oracle(nx, ny):
    b = gen.uniform_rhs(nx, ny, seed=nx * 7 + ny, ld=gen.pitch(nx, 8))
    for k in (1, 3, 6):
        x, rec = _solve(b, nx, "mg_f64", 0.0, k, variant="newcg")
        xo, io = oracle.cg_ppcg(b, tol=0.0, maxit=k, nx=nx)
        assert rec["iters"] == io["iters"], (k, rec, io)
        assert rec["status"] == io["status"], (k, rec, io)
        assert _rel(x, xo[:, :nx]) <= 1e-11, (k, _rel(x, xo[:, :nx]))


@pytest.mark.parametrize("precision", ["mg_f64"])
@pytest.mark.parametrize("nx,ny", [(100, 100), (513, 130)])
def test_pipelined_converged_matches_oracle(precision, nx, ny):
    tol = 1e-10
    b = gen.uniform_rhs(nx, ny, seed=nx + 9 * ny, ld=gen.pitch(nx, 8))
    x, rec = _solve(b, nx, precision, tol, 500, variant="newcg")
    _, io = oracle.cg_ppcg(b, tol=tol, maxit=500, nx=nx)
    assert rec["status"] == lap5cg.OK, rec
    # the pipelined recurrences stop on their recursive residual; the true one stays close
    assert rec["relres_true"] <= 3 * tol
    assert abs(rec["iters"] - io["iters"]) <= (2 if precision == "mg_f64" else 4), (rec, io)
    xt, _ = oracle.cg_pcg(b, tol=1e-13, maxit=500, nx=nx)
    assert _rel(x, xt[:, :nx]) <= gen.condition_number(nx, ny) * 3 * tol


def test_pipelined_with_binary32_vcycle_is_rejected():
    # the pipelined recurrences need an exactly linear M (a binary32 V-cycle
    # breaks them down near 1e-6, also in a binary64 restatement)
    with pytest.raises(lap5cg.Lap5cgError):
        lap5cg.cg_solve(_dev(gen.uniform_rhs(64, 64, seed=1)), tol=1e-10, precision="mg_f32", variant="newcg")


def test_pipelined_full_size_4096():
    n = 4096
    b = gen.manufactured_rhs(n, n, seed=2)
    x, rec = _solve(b, n, "mg_f64", 1e-10, 200, variant="newcg")
    assert rec["status"] == lap5cg.OK and rec["iters"] <= 30, rec
    res = b - oracle.lap5_apply(x)
    assert np.linalg.norm(res) <= 3e-10 * np.linalg.norm(b)


@pytest.mark.parametrize("variant", ["classic", "newcg"])
def test_unaligned_pitch_is_staged(variant):
    # an odd pitch goes through the aligned staging copies; same solve
    nx, ny = 100, 70
    b = gen.uniform_rhs(nx, ny, seed=23, ld=nx + 1)
    x1, r1 = _solve(b, nx, "mg_f64", 1e-10, 200, variant=variant)
    b2 = np.zeros((ny, 104))
    b2[:, :nx] = b[:, :nx]
    x2, r2 = _solve(b2, nx, "mg_f64", 1e-10, 200, variant=variant)
    assert r1["status"] == r2["status"] == lap5cg.OK
    assert r1["iters"] == r2["iters"]
    assert _rel(x1, x2) <= 1e-13


# ---------------------------------------------------------------------------
# The classic form runs as a cached CUDA graph; under stream capture it runs as
# the persistent kernel.  Both track the oracle.
# ---------------------------------------------------------------------------
def _ws_for(nx, ny, ld, precision="mg_f64", nrhs=1):
    return torch.empty(lap5cg.workspace_size(nx, ny, ld, "classic", precision, nrhs), dtype=torch.uint8,
                       device="cuda")


def test_release_graphs_then_rebuild_gives_the_same_bits():
    # a cached graph freed (once idle, once while its solve is still running)
    # and built again on the next call: the same kernels, so the same bits
    nx, ny = 300, 200
    ld = gen.pitch(nx, 8)
    b = _dev(gen.uniform_rhs(nx, ny, seed=83, ld=ld))
    ws = _ws_for(nx, ny, ld, "mg_f32")
    info = torch.empty(lap5cg.INFO_BYTES, dtype=torch.uint8, device="cuda")
    outs = []
    for release in ("none", "idle", "running"):
        x = torch.zeros((ny, ld), dtype=torch.float64, device="cuda")
        if release == "idle":
            torch.cuda.synchronize()
            lap5cg.release_graphs()
        lap5cg.cg_solve(b, tol=1e-10, maxit=500, precision="mg_f32", nx=nx, workspace=ws, info=info, out=x)
        if release == "running":
            lap5cg.release_graphs()  # the graph is in flight: the driver frees it on completion
        torch.cuda.synchronize()
        rec = lap5cg.decode_info(info)[0]
        assert rec["status"] == lap5cg.OK and rec["relres_true"] <= 1.5e-10, rec
        outs.append(x.cpu().numpy())
    assert np.array_equal(outs[0], outs[1]) and np.array_equal(outs[0], outs[2])
    lap5cg.release_graphs()
    x, info2 = lap5cg.cg_solve(b, tol=1e-10, maxit=500, precision="mg_f32", nx=nx, workspace=ws)
    assert np.array_equal(x.cpu().numpy()[:, :nx], outs[0][:, :nx])


def test_cached_graph_rebinds_rhs_solution_and_limits():
    # one workspace, so every call below hits the same cached graph: the
    # right-hand side, the solution buffer, tol and maxit change per call
    nx, ny = 300, 200
    ld = gen.pitch(nx, 8)
    ws = _ws_for(nx, ny, ld)
    bs = [gen.uniform_rhs(nx, ny, seed=s, ld=ld) for s in (31, 32)]
    runs = [(0, 0.0, 4), (1, 0.0, 6), (0, 1e-6, 500), (0, 0.0, 4)]
    first = None
    for which, tol, k in runs:
        out = torch.zeros((ny, ld), dtype=torch.float64, device="cuda")
        x, info = lap5cg.cg_solve(_dev(bs[which]), tol=tol, maxit=k, precision="mg_f64", nx=nx, workspace=ws, out=out)
        rec = lap5cg.decode_info(info)[0]
        xo, io = oracle.cg_pcg(bs[which], tol=tol, maxit=k, nx=nx)
        assert rec["iters"] == io["iters"] and rec["status"] == io["status"], (which, tol, k, rec, io)
        xg = x.cpu().numpy()[:, :nx]
        assert _rel(xg, xo[:, :nx]) <= 1e-11
        if first is None:
            first = xg
    np.testing.assert_array_equal(xg, first)  # the same call again: bit-identical


def test_stacked_right_hand_sides_share_one_graph():
    nx, ny, nrhs = 130, 67, 3
    ld = gen.pitch(nx, 8)
    b = np.stack([gen.uniform_rhs(nx, ny, seed=40 + k, ld=ld) for k in range(nrhs)])
    x, info = lap5cg.cg_solve(_dev(b), tol=0.0, maxit=5, precision="mg_f64", nx=nx)
    recs = lap5cg.decode_info(info)
    for k in range(nrhs):
        xo, io = oracle.cg_pcg(b[k], tol=0.0, maxit=5, nx=nx)
        assert recs[k]["iters"] == io["iters"] == 5
        assert _rel(x[k].cpu().numpy()[:, :nx], xo[:, :nx]) <= 1e-11


@pytest.mark.parametrize("precision", ["mg_f64", "mg_f32"])
def test_history_matches_oracle(precision):
    nx, ny, K = 300, 200, 8
    b = gen.uniform_rhs(nx, ny, seed=55, ld=gen.pitch(nx, 8))
    hist = torch.full((K + 1,), float("nan"), dtype=torch.float64, device="cuda")
    x, info = lap5cg.cg_solve(_dev(b), tol=0.0, maxit=K, precision=precision, nx=nx,
                              opts=lap5cg.default_opts(history=hist.data_ptr()))
    _, io, ho = oracle.cg_pcg(b, tol=0.0, maxit=K, nx=nx, history=True)
    h = hist.cpu().numpy()
    # binary64 V-cycle: same steps as the oracle; binary32: a rounded M
    np.testing.assert_allclose(h, ho, rtol=1e-9 if precision == "mg_f64" else 1e-4)


def test_captured_solve_takes_persistent_kernel_and_tracks_oracle():
    nx, ny, k = 513, 130, 5
    ld = gen.pitch(nx, 8)
    b = _dev(gen.uniform_rhs(nx, ny, seed=61, ld=ld))
    ws = _ws_for(nx, ny, ld)
    info = torch.empty(lap5cg.INFO_BYTES, dtype=torch.uint8, device="cuda")
    x = torch.zeros((ny, ld), dtype=torch.float64, device="cuda")
    eager, einfo = lap5cg.cg_solve(b, tol=0.0, maxit=k, precision="mg_f64", nx=nx)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.graph(g, stream=s):
        x.zero_()
        lap5cg.cg_solve(b, tol=0.0, maxit=k, precision="mg_f64", nx=nx, workspace=ws, info=info, out=x)
    xo, io = oracle.cg_pcg(b.cpu().numpy(), tol=0.0, maxit=k, nx=nx)
    for rep in range(2):
        x.fill_(7.0)
        g.replay()
        torch.cuda.synchronize()
        rec = lap5cg.decode_info(info)[0]
        assert rec["iters"] == io["iters"] == k and rec["status"] == io["status"]
        assert _rel(x.cpu().numpy()[:, :nx], xo[:, :nx]) <= 1e-11
    assert _rel(eager.cpu().numpy()[:, :nx], xo[:, :nx]) <= 1e-11


def test_graph_cache_eviction_keeps_results_right():
    # more shapes than the cache holds, then the first one again
    shapes = [(100 + 8 * i, 90 + 4 * i) for i in range(10)] + [(100, 90)]
    for nx, ny in shapes:
        b = gen.uniform_rhs(nx, ny, seed=nx + ny, ld=gen.pitch(nx, 8))
        x, rec = _solve(b, nx, "mg_f64", 0.0, 3)
        xo, io = oracle.cg_pcg(b, tol=0.0, maxit=3, nx=nx)
        assert rec["iters"] == io["iters"] == 3
        assert _rel(x, xo[:, :nx]) <= 1e-11


@pytest.mark.parametrize("nx,ny", [(300, 200), (513, 130)])
def test_nonzero_start_tracks_oracle(nx, ny):
    # x0 != 0 on part of the grid: the first residual takes the stencil there
    ld = gen.pitch(nx, 8)
    b = gen.uniform_rhs(nx, ny, seed=71, ld=ld)
    x0 = np.zeros_like(b)
    x0[ny // 3: ny // 2, : nx // 2] = gen.uniform_rhs(nx, ny, seed=72, ld=ld)[ny // 3: ny // 2, : nx // 2]
    for k in (1, 4):
        x, info = lap5cg.cg_solve(_dev(b), x0=_dev(x0), tol=0.0, maxit=k, precision="mg_f64", nx=nx)
        rec = lap5cg.decode_info(info)[0]
        xo, io = oracle.cg_pcg(b, x0=x0, tol=0.0, maxit=k, nx=nx)
        assert rec["iters"] == io["iters"] == k
        assert _rel(x.cpu().numpy()[:, :nx], xo[:, :nx]) <= 1e-11


@pytest.mark.parametrize("opt", [dict(mg_nu=1), dict(mg_nu=3), dict(mg_levels=2), dict(mg_levels=2, mg_coarse_sweeps=1),
                                 dict(mg_coarse_sweeps=2)])
def test_binary32_vcycle_options_converge_to_oracle(opt):
    # the binary32 V-cycle's fused passes and its first sweeps formed from b,
    # under the options that change which pass reads a level's first sweep
    nx, ny = 300, 200
    tol = 1e-10
    b = gen.uniform_rhs(nx, ny, seed=19, ld=gen.pitch(nx, 8))
    x, rec = _solve(b, nx, "mg_f32", tol, 3000, **opt)
    assert rec["status"] == lap5cg.OK and rec["relres_true"] <= 1.5 * tol, rec
    xt, _ = oracle.cg_pcg(b, tol=1e-13, maxit=500, nx=nx)
    assert _rel(x, xt[:, :nx]) <= gen.condition_number(nx, ny) * 2 * tol
    # the binary64 V-cycle with the same options: same iteration count within a few
    _, r64 = _solve(b, nx, "mg_f64", tol, 3000, **opt)
    assert abs(rec["iters"] - r64["iters"]) <= max(3, r64["iters"] // 5), (rec, r64)


@pytest.mark.parametrize("nx,ny", [(100, 100), (129, 130), (130, 129), (257, 258), (300, 200), (513, 130), (1000, 9),
                                   (385, 387)])
def test_binary32_vcycle_fixed_iterations_near_oracle(nx, ny):
    # The binary32 V-cycle (fused passes, first sweeps formed from b, levels in
    # shared memory) against the oracle's binary64 one at fixed iterations: they
    # differ by binary32 rounding only, so every element agrees to ~1e-6.  Shapes
    # whose coarse width is a multiple of 64 leave fine columns past the last
    # strip (129, 257, 385); odd and even heights leave fine rows above the last
    # coarse row.
    b = gen.uniform_rhs(nx, ny, seed=nx * 5 + ny, ld=gen.pitch(nx, 8))
    for k in (1, 2, 4):
        x, rec = _solve(b, nx, "mg_f32", 0.0, k)
        xo, io = oracle.cg_pcg(b, tol=0.0, maxit=k, nx=nx)
        assert rec["iters"] == io["iters"] == k
        assert _rel(x, xo[:, :nx]) <= 2e-5, (k, _rel(x, xo[:, :nx]))
