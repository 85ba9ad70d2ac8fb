"""cg_solve_batched: many grids of different shapes in one persistent launch
(teams = thread-block clusters pulling instances from a device queue).
Per instance the result must match the oracle exactly as a single solve does."""
import numpy as np
import pytest
import torch

import lap5_inputs as gen
import oracle
import paper_1803_03797_gb300 as lap5cg
from tests.helpers import rel_err

pytestmark = pytest.mark.gpu

SHAPES = [(1, 1), (3, 5), (16, 7), (40, 40), (64, 130), (130, 64), (100, 100), (200, 37), (33, 250), (255, 257)]


def _rel(a, b):
    return rel_err(a, b)  # norm-wise and element-wise


def _make(shapes, dtype=np.float64, seed0=100):
    es = 8 if dtype == np.float64 else 4
    out = []
    for k, (nx, ny) in enumerate(shapes):
        ld = gen.pitch(nx, es, 16 if dtype == np.float64 else 16)
        ld = ((ld + 3) // 4) * 4  # a multiple of 4 elements suits every precision
        out.append((nx, gen.uniform_rhs(nx, ny, seed=seed0 + k, ld=ld).astype(dtype)))
    return out


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _run(batch, **kw):
    bs = [torch.from_numpy(b).cuda() for _, b in batch]
    xs, info = lap5cg.cg_solve_batched(bs, nx_list=[nx for nx, _ in batch], **kw)
    torch.cuda.synchronize()
    return [x.cpu().numpy() for x in xs], lap5cg.decode_info(info)


@pytest.mark.parametrize("variant", ["classic", "newcg"])
def test_f64_batch_matches_oracle(variant):
    batch = _make(SHAPES)
    xs, recs = _run(batch, tol=1e-10, maxit=20000, variant=variant, precision="f64")
    for (nx, b), x, rec in zip(batch, xs, recs):
        xo, io = oracle.cg_solve(b, variant=variant, tol=1e-10, maxit=20000, nx=nx)
        assert rec["status"] == lap5cg.OK, rec
        assert abs(rec["iters"] - io["iters"]) <= 2, (rec, io)
        ny = b.shape[0]
        assert _rel(x[:, :nx], xo[:, :nx]) <= max(gen.condition_number(nx, ny) * max(1e-10, io["relres_true"]), 1e-12)


@pytest.mark.parametrize("variant", ["classic", "newcg"])
def test_fixed_iterations_equal_oracle_trajectory(variant):
    batch = _make(SHAPES)
    xs, recs = _run(batch, tol=0.0, maxit=25, variant=variant, precision="f64")
    for (nx, b), x, rec in zip(batch, xs, recs):
        if nx * b.shape[0] <= 50:
            continue  # past exact convergence the iterates are rounding noise
        xo, io = oracle.cg_solve(b, variant=variant, tol=0.0, maxit=25, nx=nx)
        assert rec["iters"] == io["iters"]
        assert _rel(x[:, :nx], xo[:, :nx]) <= 1e-10


@pytest.mark.parametrize("team", [1, 2, 4, 8, 16])
def test_team_sizes_agree(team):
    batch = _make(SHAPES[3:])
    opts = lap5cg.default_opts(team_ctas=team)
    xs, recs = _run(batch, tol=0.0, maxit=30, variant="classic", precision="f64", opts=opts)
    for (nx, b), x in zip(batch, xs):
        xo, _ = oracle.cg_classic(b, tol=0.0, maxit=30, nx=nx)
        assert _rel(x[:, :nx], xo[:, :nx]) <= 1e-10


def test_f32_batch():
    batch = _make(SHAPES, dtype=np.float32)
    xs, recs = _run(batch, tol=1e-5, maxit=20000, variant="classic", precision="f32")
    for (nx, b), x, rec in zip(batch, xs, recs):
        assert rec["status"] == lap5cg.OK, rec
        ny = b.shape[0]
        xo, _ = oracle.cg_classic(b.astype(np.float64), tol=1e-13, maxit=20000, nx=nx)
        assert _rel(x[:, :nx].astype(np.float64), xo[:, :nx]) <= gen.condition_number(nx, ny) * (2e-5 + 4 * 2.0 ** -24)
    xs, recs = _run(batch, tol=0.0, maxit=30, variant="newcg", precision="f32")
    for (nx, b), x, rec in zip(batch, xs, recs):
        if nx * b.shape[0] <= 60:
            continue  # past exact convergence the iterates are rounding noise
        xo, io = oracle.cg_newcg(b.astype(np.float64), tol=0.0, maxit=30, nx=nx)
        assert rec["iters"] == io["iters"]
        assert _rel(x[:, :nx].astype(np.float64), xo[:, :nx]) <= 1e-3


@pytest.mark.parametrize("precision", ["ir_f32", "ir_bf16pr"])
def test_ir_batch(precision):
    batch = _make(SHAPES)
    xs, recs = _run(batch, tol=1e-10, maxit=10 ** 6, variant="classic", precision=precision)
    for (nx, b), x, rec in zip(batch, xs, recs):
        assert rec["status"] == lap5cg.OK and rec["relres_true"] <= 1e-10, rec
        ny = b.shape[0]
        xo, _ = oracle.cg_classic(b, tol=1e-13, maxit=10 ** 6, nx=nx)
        assert _rel(x[:, :nx], xo[:, :nx]) <= max(gen.condition_number(nx, ny) * 2e-10, 1e-13)


def test_convergence_masking_and_initial_guess():
    batch = _make([(64, 64), (120, 90), (90, 120)])
    bs = [torch.from_numpy(b).cuda() for _, b in batch]
    bs[0].zero_()  # converges at once
    x_pre, _ = lap5cg.cg_solve(bs[1], tol=1e-12, maxit=20000)
    xs = [torch.ones_like(bs[0]), x_pre.clone(), torch.zeros_like(bs[2])]
    xs_out, info = lap5cg.cg_solve_batched(bs, xs=xs, tol=1e-10, maxit=20000, precision="f64")
    recs = lap5cg.decode_info(info)
    assert recs[0]["status"] == lap5cg.OK and recs[0]["iters"] == 0 and not xs_out[0].cpu().numpy().any()
    assert recs[1]["status"] == lap5cg.OK and recs[1]["iters"] == 0  # started at a solution
    xo, io = oracle.cg_classic(batch[2][1], tol=1e-10, maxit=20000)
    assert recs[2]["status"] == lap5cg.OK and abs(recs[2]["iters"] - io["iters"]) <= 2


def test_cuda_graph_capture_and_replay():
    batch = _make(SHAPES[2:])
    bs = [torch.from_numpy(b).cuda() for _, b in batch]
    nxs = [nx for nx, _ in batch]
    xs = [torch.zeros_like(b) for b in bs]
    need = lap5cg.batched_workspace_size(nxs, [b.shape[0] for b in bs], [b.shape[1] for b in bs], "classic", "ir_f32")
    ws = torch.empty(need, dtype=torch.uint8, device="cuda")
    info = torch.empty(len(bs) * lap5cg.INFO_BYTES, dtype=torch.uint8, device="cuda")
    # eager reference
    ref, ref_info = lap5cg.cg_solve_batched(bs, tol=1e-10, maxit=10 ** 6, precision="ir_f32", nx_list=nxs)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.graph(g, stream=s):
        for x in xs:
            x.zero_()
        lap5cg.cg_solve_batched(bs, xs=xs, tol=1e-10, maxit=10 ** 6, precision="ir_f32", nx_list=nxs,
                                workspace=ws, info=info)
    for rep in range(2):
        for x in xs:
            x.fill_(123.0)  # replay must reset x0 itself
        g.replay()
        torch.cuda.synchronize()
        recs = lap5cg.decode_info(info)
        assert all(r["status"] == lap5cg.OK for r in recs)
        for x, r in zip(xs, ref):
            np.testing.assert_array_equal(x.cpu().numpy(), r.cpu().numpy())


def test_batched_workload_256_ir_f32():
    nxs, nys = gen.batched_shapes(256, 64, 1024, seed=4)
    bs_np = gen.batched_rhs(nxs, nys, seed=4, elem_bytes=8, align_bytes=32)
    bs = [torch.from_numpy(b).cuda() for b in bs_np]
    xs, info = lap5cg.cg_solve_batched(bs, tol=1e-10, maxit=10 ** 7, variant="classic", precision="ir_f32",
                                       nx_list=nxs)
    recs = lap5cg.decode_info(info)
    assert all(r["status"] == lap5cg.OK and r["relres_true"] <= 1e-10 for r in recs)
    # true residuals recomputed by the oracle's stencil
    for k in range(0, 256, 17):
        x = xs[k].cpu().numpy()
        b = bs_np[k]
        nx = nxs[k]
        res = b[:, :nx] - oracle.lap5_apply(x, nx=nx)[:, :nx]
        assert np.linalg.norm(res) <= 1.5e-10 * np.linalg.norm(b[:, :nx])
    # the smallest instances against the FP64 oracle solution
    small = sorted(range(256), key=lambda k: nxs[k] * nys[k])[:3]
    for k in small:
        xo, _ = oracle.cg_classic(bs_np[k], tol=1e-13, maxit=10 ** 6, nx=nxs[k])
        nx = nxs[k]
        assert _rel(xs[k].cpu().numpy()[:, :nx], xo[:, :nx]) <= gen.condition_number(nx, nys[k]) * 2e-10


def test_batched_invalid_arguments():
    b = torch.zeros((8, 7), dtype=torch.float64, device="cuda")  # ld 7 is not a multiple of 2
    with pytest.raises(lap5cg.Lap5cgError):
        lap5cg.cg_solve_batched([b], tol=1e-8, maxit=10, precision="f64")
    b = torch.zeros((8, 8), dtype=torch.float64, device="cuda")
    with pytest.raises(lap5cg.Lap5cgError):
        lap5cg.cg_solve_batched([b], tol=1e-8, maxit=10, precision="ir_f32", variant="newcg")


@pytest.mark.parametrize("variant", ["classic", "newcg"])
def test_batched_small_instances_take_the_resident_kernel(variant):
    # 100 instances that fit in one cluster's shared memory (two launches of
    # the cluster-resident kernel, 96 a launch) mixed with three that do not
    # (the persistent kernel): every one against the oracle, in caller order
    rng = np.random.default_rng(17)
    shapes = [(int(rng.integers(16, 90)), int(rng.integers(16, 90))) for _ in range(100)]
    shapes[10:10] = [(700, 300), (300, 700), (1100, 90)]
    bs = []
    for k, (nx, ny) in enumerate(shapes):
        bs.append(gen.uniform_rhs(nx, ny, seed=500 + k, ld=gen.pitch(nx, 8, 32)))
    xs, info = lap5cg.cg_solve_batched([_dev(b) for b in bs], tol=1e-10, maxit=100000, variant=variant,
                                       precision="f64", nx_list=[s[0] for s in shapes])
    recs = lap5cg.decode_info(info)
    for k, (nx, ny) in enumerate(shapes):
        xo, io = oracle.cg_solve(bs[k], variant=variant, tol=1e-10, maxit=100000, nx=nx)
        rec = recs[k]
        assert rec["status"] == lap5cg.OK, (k, rec)
        assert abs(rec["iters"] - io["iters"]) <= 2, (k, rec, io)
        kappa = gen.condition_number(nx, ny)
        assert _rel(xs[k].cpu().numpy()[:, :nx], xo[:, :nx]) <= kappa * max(1e-10, io["relres_true"]), k


def test_batched_one_small_instance_is_as_fast_as_a_single_solve():
    # the paper's 100 x 100 grid through cg_solve_batched takes the same
    # cluster-resident kernel as cg_solve: within 1.5x of its time
    b = _dev(gen.uniform_rhs(100, 100, seed=1))
    times = {}
    for path in ("single", "batched"):
        def run():
            if path == "single":
                return lap5cg.cg_solve(b, tol=1e-8, maxit=10000, variant="newcg")[1]
            return lap5cg.cg_solve_batched([b], tol=1e-8, maxit=10000, variant="newcg", precision="f64")[1]
        run()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(10):
            info = run()
        e1.record()
        torch.cuda.synchronize()
        assert lap5cg.decode_info(info)[0]["status"] == lap5cg.OK
        times[path] = e0.elapsed_time(e1) / 10
    assert times["batched"] <= 1.5 * times["single"], times
