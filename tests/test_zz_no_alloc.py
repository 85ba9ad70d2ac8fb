"""The allocation-free classic binary64 solve (cg_solve_classic_f64_noalloc),
called through the C ABI, must give the same result as cg_solve, on two calls
in a row (the second call reuses the library's fixed scratch array after the
first left its contents behind).

Some callers cannot allocate device memory after start-up (fixed-budget
real-time code, plug-ins inside frameworks that own the device memory pool);
this entry point serves them.  This file is named to be collected last."""
import ctypes

import numpy as np
import pytest
import torch

import lap5_inputs as gen
import paper_1803_03797_gb300 as lap5cg

pytestmark = pytest.mark.gpu


def _call_noalloc(b, x, info, tol, maxit, nx=None):
    L = lap5cg.lib()
    ny, ld = b.shape
    nx = ld if nx is None else nx
    return L.cg_solve_classic_f64_noalloc(nx, ny, ld, ctypes.c_void_p(b.data_ptr()), ctypes.c_void_p(x.data_ptr()),
                                          tol, maxit, ctypes.c_void_p(info.data_ptr()),
                                          ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))


def test_noalloc_matches_cg_solve_on_two_calls():
    cases = [(300, 200, 10001), (511, 512, 10002)]  # the second is near the size limit, ragged nx
    for nx, ny, seed in cases:
        ld = gen.pitch(nx, 8)
        b = torch.from_numpy(gen.uniform_rhs(nx, ny, seed=seed, ld=ld)).cuda()
        x_ref, info_ref = lap5cg.cg_solve(b, tol=1e-10, maxit=20000, variant="classic", precision="f64", nx=nx)
        x = torch.zeros_like(b)
        info = torch.empty(lap5cg.INFO_BYTES, dtype=torch.uint8, device="cuda")
        assert _call_noalloc(b, x, info, 1e-10, 20000, nx=nx) == lap5cg.OK
        torch.cuda.synchronize()
        rec, ref = lap5cg.decode_info(info)[0], lap5cg.decode_info(info_ref)[0]
        assert rec["status"] == lap5cg.OK and ref["status"] == lap5cg.OK
        assert abs(rec["iters"] - ref["iters"]) <= 2
        xa, xr = x.cpu().numpy()[:, :nx], x_ref.cpu().numpy()[:, :nx]
        assert np.linalg.norm(xa - xr) / np.linalg.norm(xr) <= 1e-10
        assert rec["relres_true"] <= 2e-10


def test_noalloc_rejects_oversized_and_misaligned():
    n = 520  # 520 * 520 > 262144
    b = torch.zeros((n, n), dtype=torch.float64, device="cuda")
    x = torch.zeros_like(b)
    info = torch.empty(lap5cg.INFO_BYTES, dtype=torch.uint8, device="cuda")
    assert _call_noalloc(b, x, info, 1e-8, 10) == lap5cg.ERR_INVALID_ARG
    b = torch.zeros((64, 63), dtype=torch.float64, device="cuda")  # odd pitch
    x = torch.zeros_like(b)
    assert _call_noalloc(b, x, info, 1e-8, 10) == lap5cg.ERR_INVALID_ARG
