"""Memory-safety checks without a sanitizer: guard bands and poisoned padding.

Every buffer a solve touches -- b, x, the workspace, the info records -- is a
view into a larger allocation filled with a canary byte; after the solve the
bands around each view must be untouched.  The padding columns of b and x
(columns nx .. ld-1) hold NaN: a kernel may read them (vector loads mask them
afterwards) but they must not reach the result, and the padding of x must not
be written.  The solution must equal, bit for bit, the same solve on clean
buffers."""
import numpy as np
import pytest
import torch

import lap5_inputs as gen
import paper_1803_03797_gb300 as lap5cg

pytestmark = pytest.mark.gpu

G = 4096      # guard bytes on each side
CANARY = 0xA5


def _guarded(nbytes):
    buf = torch.full((nbytes + 2 * G,), CANARY, dtype=torch.uint8, device="cuda")
    return buf, buf[G:G + nbytes]


def _intact(buf, nbytes):
    return bool((buf[:G] == CANARY).all()) and bool((buf[G + nbytes:] == CANARY).all())


def _grid_view(raw, shape, dtype):
    return raw.view(dtype).view(shape)


CASES = [
    ("f64", "classic", {}), ("f64", "newcg", {}), ("f64", "classic", {"reproducible": 1}),
    ("f64", "classic", {"resident": -1, "ring_slots": -1}), ("f64", "classic", {"lane_vec": 4, "ring_slots": 4}),
    ("f32", "classic", {}), ("f32", "classic", {"lane_vec": 8, "ring_slots": 4}),
    ("ir_f32", "classic", {}), ("ir_bf16pr", "classic", {}), ("mg_f32", "classic", {}), ("mg_f64", "newcg", {}),
]
SHAPES = [(100, 37, 101), (257, 130, 260), (1030, 70, 1032), (64, 64, 64), (1, 9, 4)]


@pytest.mark.parametrize("precision,variant,opt", CASES)
@pytest.mark.parametrize("nx,ny,ld", SHAPES)
def test_guard_bands_and_poisoned_padding(precision, variant, opt, nx, ny, ld):
    dtype = torch.float32 if precision == "f32" else torch.float64
    es = 4 if dtype == torch.float32 else 8
    tol, maxit = (1e-5, 300) if precision == "f32" else (1e-10, 300)
    b_np = gen.uniform_rhs(nx, ny, seed=nx + ny, ld=ld)
    opts = lap5cg.default_opts(**opt)
    # the clean reference solve
    b_clean = torch.from_numpy(b_np).to("cuda", dtype)
    x_ref, info_ref = lap5cg.cg_solve(b_clean, tol=tol, maxit=maxit, variant=variant, precision=precision, nx=nx,
                                      opts=opts)
    # the guarded solve
    nb = ny * ld * es
    bbuf, braw = _guarded(nb)
    xbuf, xraw = _guarded(nb)
    need = lap5cg.workspace_size(nx, ny, ld, variant, precision)
    wbuf, wraw = _guarded(need)
    ibuf, iraw = _guarded(lap5cg.INFO_BYTES)
    b = _grid_view(braw, (ny, ld), dtype)
    x = _grid_view(xraw, (ny, ld), dtype)
    b.copy_(b_clean)
    b[:, nx:] = float("nan")
    x.zero_()
    x[:, nx:] = float("nan")
    b_before = b.clone()
    x_out, info = lap5cg.cg_solve(b, x0=x, out=x, tol=tol, maxit=maxit, variant=variant, precision=precision,
                                  nx=nx, opts=opts, workspace=wraw, info=iraw)
    torch.cuda.synchronize()
    for buf, n, name in ((bbuf, nb, "b"), (xbuf, nb, "x"), (wbuf, need, "workspace"), (ibuf, lap5cg.INFO_BYTES, "info")):
        assert _intact(buf, n), "guard band around %s overwritten" % name
    assert torch.equal(b[:, :nx], b_before[:, :nx]) and torch.isnan(b[:, nx:]).all(), "b was written"
    assert torch.isnan(x[:, nx:]).all(), "padding columns of x were written"
    rec, rec_ref = lap5cg.decode_info(info)[0], lap5cg.decode_info(info_ref)[0]
    assert rec["status"] == rec_ref["status"] and rec["iters"] == rec_ref["iters"], (rec, rec_ref)
    assert torch.equal(x[:, :nx], x_ref[:, :nx]), "padding values reached the solution"


def test_guard_bands_batched():
    shapes = [(100, 37, 104), (257, 130, 260), (64, 64, 64)]
    for precision in ("ir_f32", "f64"):
        bufs, bs, xs = [], [], []
        for k, (nx, ny, ld) in enumerate(shapes):
            nb = ny * ld * 8
            bbuf, braw = _guarded(nb)
            xbuf, xraw = _guarded(nb)
            b = _grid_view(braw, (ny, ld), torch.float64)
            x = _grid_view(xraw, (ny, ld), torch.float64)
            b.copy_(torch.from_numpy(gen.uniform_rhs(nx, ny, seed=k, ld=ld)))
            b[:, nx:] = float("nan")
            x.zero_()
            x[:, nx:] = float("nan")
            bufs += [(bbuf, nb, "b%d" % k), (xbuf, nb, "x%d" % k)]
            bs.append(b)
            xs.append(x)
        nxs = [s[0] for s in shapes]
        need = lap5cg.batched_workspace_size(nxs, [s[1] for s in shapes], [s[2] for s in shapes], "classic", precision)
        wbuf, wraw = _guarded(need)
        xs_out, info = lap5cg.cg_solve_batched(bs, xs=xs, tol=1e-10, maxit=10 ** 6, precision=precision, nx_list=nxs,
                                               workspace=wraw)
        torch.cuda.synchronize()
        for buf, n, name in bufs + [(wbuf, need, "workspace")]:
            assert _intact(buf, n), "guard band around %s overwritten (%s)" % (name, precision)
        for (nx, ny, ld), b, x in zip(shapes, bs, xs):
            assert torch.isnan(b[:, nx:]).all() and torch.isnan(x[:, nx:]).all()
            assert torch.isfinite(x[:, :nx]).all()
        assert all(r["status"] == lap5cg.OK for r in lap5cg.decode_info(info))


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32, torch.bfloat16])
@pytest.mark.parametrize("nx,ny,ld", [(100, 37, 104), (257, 130, 260), (1030, 70, 1032), (63, 5, 63), (1, 9, 4)])
def test_guard_bands_lap5_apply(dtype, nx, ny, ld):
    es = torch.tensor([], dtype=dtype).element_size()
    nb = ny * ld * es
    xbuf, xraw = _guarded(nb)
    ybuf, yraw = _guarded(nb)
    x = xraw.view(dtype).view(ny, ld)
    y = yraw.view(dtype).view(ny, ld)
    x.copy_(torch.from_numpy(gen.uniform_rhs(nx, ny, seed=nx + ny, ld=ld)).to("cuda", dtype))
    x[:, nx:] = float("nan")
    y.fill_(7.0)
    ref = lap5cg.lap5_apply(x[:, :nx].contiguous())
    lap5cg.lap5_apply(x, nx=nx, out=y)
    torch.cuda.synchronize()
    assert _intact(xbuf, nb) and _intact(ybuf, nb), "guard band overwritten"
    assert (y[:, nx:] == 7.0).all(), "padding columns of y were written"
    assert torch.equal(y[:, :nx], ref), "padding values reached the result"
