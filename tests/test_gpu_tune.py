"""The autotuner changes launch parameters only: solves with the options it
returns must still match the oracle, and its cache round-trips."""
import numpy as np
import pytest
import torch

import lap5_inputs as gen
import oracle
import paper_1803_03797_gb300 as lap5cg
from tests.helpers import rel_err

pytestmark = pytest.mark.gpu


def _rel(a, b):
    return rel_err(a, b)  # norm-wise and element-wise


@pytest.mark.parametrize("variant,precision", [("classic", "f64"), ("newcg", "f64"), ("classic", "f32"),
                                               ("classic", "ir_f32")])
def test_autotune_single(tmp_path, monkeypatch, variant, precision):
    monkeypatch.setenv("LAP5CG_TUNE_CACHE", str(tmp_path / "tune.json"))
    n = 384
    dt = np.float32 if precision == "f32" else np.float64
    b_np = gen.uniform_rhs(n, n, seed=3).astype(dt)
    b = torch.from_numpy(b_np).cuda()
    opts, ms = lap5cg.autotune(b, variant=variant, precision=precision, iters=30)
    assert ms > 0
    cached = lap5cg.tuned_opts(n, n, variant, precision)
    assert cached is not None
    for f in ("warps_per_cta", "ring_slots", "min_rows", "store_z"):
        assert getattr(cached, f) == getattr(opts, f)
    if precision.startswith("ir"):
        x, info = lap5cg.cg_solve(b, tol=1e-10, maxit=10 ** 6, variant=variant, precision=precision, opts=opts)
        rec = lap5cg.decode_info(info)[0]
        assert rec["status"] == lap5cg.OK and rec["relres_true"] <= 1e-10
        return
    x, info = lap5cg.cg_solve(b, tol=0.0, maxit=25, variant=variant, precision=precision, opts=opts)
    xo, _ = oracle.cg_solve(b_np.astype(np.float64), variant=variant, tol=0.0, maxit=25)
    assert _rel(x.cpu().numpy().astype(np.float64), xo) <= (1e-10 if precision == "f64" else 1e-4)


def test_autotune_batched(tmp_path, monkeypatch):
    monkeypatch.setenv("LAP5CG_TUNE_CACHE", str(tmp_path / "tune.json"))
    # the small instances go to the cluster-resident kernel, the two large ones
    # to the team kernel whose team size the tuner sweeps
    shapes = [(64, 200), (300, 120), (150, 150), (96, 64), (256, 256), (128, 300), (700, 640), (900, 500)]
    bs_np = [gen.uniform_rhs(nx, ny, seed=10 + k, ld=gen.pitch(nx, 8, 32)) for k, (nx, ny) in enumerate(shapes)]
    bs = [torch.from_numpy(b).cuda() for b in bs_np]
    nxs = [nx for nx, _ in shapes]
    opts, ms = lap5cg.autotune_batched(bs, variant="classic", precision="f64", iters=30, nx_list=nxs)
    # 0 keeps the automatic team size when no candidate is faster
    assert ms > 0 and opts.team_ctas in (0, 1, 2, 4, 8, 16)
    xs, info = lap5cg.cg_solve_batched(bs, tol=0.0, maxit=25, precision="f64", nx_list=nxs, opts=opts)
    for k, (nx, ny) in enumerate(shapes):
        xo, _ = oracle.cg_classic(bs_np[k], tol=0.0, maxit=25, nx=nx)
        assert _rel(xs[k].cpu().numpy()[:, :nx], xo[:, :nx]) <= 1e-10
