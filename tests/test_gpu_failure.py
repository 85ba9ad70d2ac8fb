"""Failure detection without a GPU fault: device waits are bounded and end in a
status the host reads; the context stays usable afterwards.  Inputs that make a
reduction non-finite are host-made faults."""
import numpy as np
import pytest
import torch

import lap5_inputs as gen
import paper_1803_03797_gb300 as lap5cg

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("variant", ["classic", "newcg"])
def test_grid_barrier_time_limit_ends_in_a_status(variant):
    # A 100 ns barrier limit that the waits between passes exceed.  Rows are
    # loaded straight into registers here (no asynchronous copies in flight),
    # so every CTA leaves at its next barrier check.
    # 2048^2: a pass takes ~0.1 ms, so CTAs reach each barrier microseconds apart
    b = torch.from_numpy(gen.uniform_rhs(2048, 2048, seed=1)).cuda()
    opts = lap5cg.default_opts(timeout_s=1e-7, ring_slots=-1)
    x, info = lap5cg.cg_solve(b, tol=1e-10, maxit=200, variant=variant, opts=opts)
    rec = lap5cg.decode_info(info)[0]
    assert rec["status"] == lap5cg.ERR_SYNC_TIMEOUT, rec
    # the context is still usable
    x2, info2 = lap5cg.cg_solve(b, tol=1e-6, maxit=20000, variant=variant)
    assert lap5cg.decode_info(info2)[0]["status"] == lap5cg.OK


@pytest.mark.parametrize("precision", ["f64", "ir_f32"])
def test_nonfinite_input_in_the_middle_of_a_batch(precision):
    shapes = [(64, 64), (100, 80), (80, 100)]
    bs = [torch.from_numpy(gen.uniform_rhs(nx, ny, seed=k, ld=gen.pitch(nx, 8, 32))).cuda()
          for k, (nx, ny) in enumerate(shapes)]
    bs[1][10, 10] = float("nan")
    xs, info = lap5cg.cg_solve_batched(bs, tol=1e-10, maxit=10 ** 6, precision=precision,
                                       nx_list=[nx for nx, _ in shapes])
    recs = lap5cg.decode_info(info)
    assert recs[1]["status"] == lap5cg.ERR_NONFINITE
    assert recs[0]["status"] == lap5cg.OK and recs[2]["status"] == lap5cg.OK
    assert np.isfinite(xs[0].cpu().numpy()).all() and np.isfinite(xs[2].cpu().numpy()).all()
