"""The allocation-free classic binary64 solve (cg_solve_classic_f64_noalloc),
called through the C ABI, must give the same result as cg_solve, on two calls
in a row (the second call reuses the library's fixed scratch array after the
first left its contents behind), and the same iterates as the oracle's
Algorithm 1 at a fixed iteration count.

Some callers cannot allocate device memory after start-up (fixed-budget
real-time code, plug-ins inside frameworks that own the device memory pool);
this entry point serves them.  This file is named to be collected last."""
import ctypes

import numpy as np
import pytest
import torch

import lap5_inputs as gen
import oracle
import paper_1803_03797_gb300 as lap5cg

pytestmark = pytest.mark.gpu


def _call_noalloc(b, x, info, tol, maxit, nx=None, ny=None, ld=None):
    L = lap5cg.lib()
    ny = b.shape[0] if ny is None else ny
    ld = b.shape[-1] if ld is None else ld
    nx = ld if nx is None else nx
    return L.cg_solve_classic_f64_noalloc(nx, ny, ld, ctypes.c_void_p(b.data_ptr()), ctypes.c_void_p(x.data_ptr()),
                                          tol, maxit, ctypes.c_void_p(info.data_ptr()),
                                          ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))


def _info():
    return torch.empty(lap5cg.INFO_BYTES, dtype=torch.uint8, device="cuda")


def test_noalloc_matches_cg_solve_on_two_calls():
    cases = [(300, 200, 10001), (511, 512, 10002)]  # the second is near the size limit, ragged nx
    for nx, ny, seed in cases:
        ld = gen.pitch(nx, 8)
        b = torch.from_numpy(gen.uniform_rhs(nx, ny, seed=seed, ld=ld)).cuda()
        x_ref, info_ref = lap5cg.cg_solve(b, tol=1e-10, maxit=20000, variant="classic", precision="f64", nx=nx)
        x = torch.zeros_like(b)
        info = _info()
        assert _call_noalloc(b, x, info, 1e-10, 20000, nx=nx) == lap5cg.OK
        torch.cuda.synchronize()
        rec, ref = lap5cg.decode_info(info)[0], lap5cg.decode_info(info_ref)[0]
        assert rec["status"] == lap5cg.OK and ref["status"] == lap5cg.OK
        assert abs(rec["iters"] - ref["iters"]) <= 2
        xa, xr = x.cpu().numpy()[:, :nx], x_ref.cpu().numpy()[:, :nx]
        assert np.linalg.norm(xa - xr) / np.linalg.norm(xr) <= 1e-10
        assert np.max(np.abs(xa - xr)) <= 1e-10 * np.max(np.abs(xr))
        assert rec["relres_true"] <= 2e-10


def test_noalloc_matches_oracle_at_fixed_iterations():
    # Algorithm 1 at k = 60 updates (tol 0): element-wise against the oracle's
    # iterate, on two calls in a row with different grids
    for nx, ny, seed in [(257, 190, 10011), (96, 512, 10012)]:
        ld = gen.pitch(nx, 8)
        bh = gen.uniform_rhs(nx, ny, seed=seed, ld=ld)
        b = torch.from_numpy(bh).cuda()
        x = torch.zeros_like(b)
        info = _info()
        assert _call_noalloc(b, x, info, 0.0, 60, nx=nx) == lap5cg.OK
        torch.cuda.synchronize()
        rec = lap5cg.decode_info(info)[0]
        xo, io = oracle.cg_classic(bh, tol=0.0, maxit=60, nx=nx)
        assert rec["status"] == lap5cg.NOT_CONVERGED and rec["iters"] == io["iters"] == 60
        xa, xr = x.cpu().numpy()[:, :nx], xo[:, :nx]
        assert np.max(np.abs(xa - xr)) <= 1e-10 * np.max(np.abs(xr))


def test_noalloc_wrapper_with_initial_guess():
    nx, ny = 200, 150
    ld = gen.pitch(nx, 8)
    b = torch.from_numpy(gen.uniform_rhs(nx, ny, seed=10021, ld=ld)).cuda()
    x0 = torch.from_numpy(gen.uniform_rhs(nx, ny, seed=10022, ld=ld)).cuda()
    x, info = lap5cg.cg_solve_classic_f64_noalloc(b, x0=x0, tol=1e-10, maxit=20000, nx=nx)
    xr, ir = lap5cg.cg_solve(b, x0=x0, tol=1e-10, maxit=20000, variant="classic", precision="f64", nx=nx,
                             opts=lap5cg.default_opts(resident=-1))
    rec, ref = lap5cg.decode_info(info)[0], lap5cg.decode_info(ir)[0]
    assert rec["status"] == lap5cg.OK and ref["status"] == lap5cg.OK
    assert abs(rec["iters"] - ref["iters"]) <= 2
    xa, xb = x.cpu().numpy()[:, :nx], xr.cpu().numpy()[:, :nx]
    assert np.max(np.abs(xa - xb)) <= 1e-10 * np.max(np.abs(xb))
    # the wrapper rejects mismatched outputs before any launch
    with pytest.raises(ValueError):
        lap5cg.cg_solve_classic_f64_noalloc(b, out=torch.zeros_like(b, dtype=torch.float32))
    with pytest.raises(ValueError):
        lap5cg.cg_solve_classic_f64_noalloc(b, x0=x0[:, :-8].contiguous())
    with pytest.raises(ValueError):
        lap5cg.cg_solve_classic_f64_noalloc(b, info=torch.empty(8, dtype=torch.uint8, device="cuda"))


def test_noalloc_rejects_oversized_misaligned_and_overlapping():
    info = _info()
    n = 520  # 520 * 520 > 262144
    b = torch.zeros((n, n), dtype=torch.float64, device="cuda")
    x = torch.zeros_like(b)
    assert _call_noalloc(b, x, info, 1e-8, 10) == lap5cg.ERR_INVALID_ARG
    b = torch.zeros((64, 63), dtype=torch.float64, device="cuda")  # odd pitch
    x = torch.zeros_like(b)
    assert _call_noalloc(b, x, info, 1e-8, 10) == lap5cg.ERR_INVALID_ARG
    # b or x 8 bytes off a 16-byte boundary
    big = torch.zeros(64 * 64 + 2, dtype=torch.float64, device="cuda")
    good = torch.zeros(64 * 64, dtype=torch.float64, device="cuda")
    off = big[1:1 + 64 * 64]
    assert off.data_ptr() % 16 == 8
    assert _call_noalloc(off, good, info, 1e-8, 10, ny=64, ld=64) == lap5cg.ERR_INVALID_ARG
    assert _call_noalloc(good, off, info, 1e-8, 10, ny=64, ld=64) == lap5cg.ERR_INVALID_ARG
    # overlapping b and x
    buf = torch.zeros(2 * 64 * 64, dtype=torch.float64, device="cuda")
    assert _call_noalloc(buf[:64 * 64], buf[32 * 64:96 * 64], info, 1e-8, 10, ny=64, ld=64) == lap5cg.ERR_INVALID_ARG
    assert _call_noalloc(buf[:64 * 64], buf[:64 * 64], info, 1e-8, 10, ny=64, ld=64) == lap5cg.ERR_INVALID_ARG
    # nothing was launched: the context is fine and a valid call still works
    bh = gen.uniform_rhs(64, 64, seed=10031, ld=64)
    b = torch.from_numpy(bh).cuda()
    x = torch.zeros_like(b)
    assert _call_noalloc(b, x, info, 1e-10, 1000) == lap5cg.OK
    torch.cuda.synchronize()
    assert lap5cg.decode_info(info)[0]["status"] == lap5cg.OK
