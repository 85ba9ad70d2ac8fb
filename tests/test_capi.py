"""CPU-side checks of the C ABI: the library builds, loads, exports every
function include/lap5cg.h declares, and rejects invalid arguments on the host
(before any CUDA call)."""
import ctypes
import glob
import os
import re

import pytest

import paper_1803_03797_gb300 as lap5cg

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        names.update(re.findall(r"LAP5CG_API\s+[\w\s\*]+?\b(\w+)\s*\(", text))
    return sorted(names)


def test_header_declares_the_boundary():
    names = declared_functions()
    for n in ("lap5_apply", "cg_workspace_size", "cg_solve", "cg_solve_batched", "lap5cg_status_string"):
        assert n in names


def test_library_exports_every_declared_symbol():
    L = lap5cg.lib()
    for n in declared_functions():
        assert hasattr(L, n), n
    assert set(lap5cg.EXPORTED) <= set(declared_functions())


def test_release_graphs_with_an_empty_cache():
    # no graph has been built in this process: nothing to free, no device needed
    assert lap5cg.lib().lap5cg_release_graphs() == lap5cg.OK


def test_status_strings():
    for code in (0, 1, -1, -2, -3, -4, -5, -6, -7):
        assert lap5cg.status_string(code) != "unknown status"
    assert lap5cg.status_string(99) == "unknown status"


def test_default_opts():
    o = lap5cg.default_opts()
    assert o.store_z == -1 and o.true_residual == 1 and o.rr_period == 0 and not o.history


def test_workspace_size_host_logic():
    f64 = lap5cg.workspace_size(100, 100, 100, "classic", "f64")
    assert f64 > 4 * 100 * 100 * 8
    assert lap5cg.workspace_size(100, 100, 100, "newcg", "f64") > f64
    assert lap5cg.workspace_size(100, 100, 100, "classic", "f32") < f64
    # an odd pitch needs staging buffers
    assert lap5cg.workspace_size(101, 100, 101, "classic", "f64") > lap5cg.workspace_size(101, 100, 102, "classic", "f64")
    for bad in [(0, 5, 5), (5, 0, 5), (5, 5, 4)]:
        assert lap5cg.workspace_size(*bad, "classic", "f64") == 0


def test_invalid_arguments_rejected_before_launch():
    L = lap5cg.lib()
    vp = ctypes.c_void_p
    dummy = vp(1 << 20)
    # lap5_apply: bad shape / dtype / null
    assert L.lap5_apply(0, 4, 4, 0, dummy, vp(2 << 20), None) == lap5cg.ERR_INVALID_ARG
    assert L.lap5_apply(4, 4, 3, 0, dummy, vp(2 << 20), None) == lap5cg.ERR_INVALID_ARG
    assert L.lap5_apply(4, 4, 4, 7, dummy, vp(2 << 20), None) == lap5cg.ERR_INVALID_ARG
    assert L.lap5_apply(4, 4, 4, 0, None, vp(2 << 20), None) == lap5cg.ERR_INVALID_ARG
    assert L.lap5_apply(4, 4, 4, 0, dummy, dummy, None) == lap5cg.ERR_INVALID_ARG  # overlap
    ws = vp(16 << 20)
    info = vp(32 << 20)
    big = 1 << 26
    args = dict(nx=8, ny=8, ld=8, b=vp(1 << 20), x=vp(2 << 20), tol=1e-8, maxit=10, variant=0, precision=0, nrhs=1,
                ws=ws, wsb=big, info=info)

    def call(**kw):
        a = dict(args)
        a.update(kw)
        return L.cg_solve(a["nx"], a["ny"], a["ld"], a["b"], a["x"], a["tol"], a["maxit"], a["variant"],
                          a["precision"], a["nrhs"], a["ws"], a["wsb"], a["info"], None, None)

    assert call(nx=0) == lap5cg.ERR_INVALID_ARG
    assert call(ld=7) == lap5cg.ERR_INVALID_ARG
    assert call(maxit=-1) == lap5cg.ERR_INVALID_ARG
    assert call(variant=5) == lap5cg.ERR_INVALID_ARG
    assert call(precision=9) == lap5cg.ERR_INVALID_ARG
    assert call(nrhs=0) == lap5cg.ERR_INVALID_ARG
    assert call(b=None) == lap5cg.ERR_INVALID_ARG
    assert call(info=None) == lap5cg.ERR_INVALID_ARG
    assert call(tol=float("nan")) == lap5cg.ERR_INVALID_ARG
    assert call(x=vp((1 << 20) + 64)) == lap5cg.ERR_INVALID_ARG  # b and x overlap
    assert call(wsb=16) == lap5cg.ERR_WORKSPACE
    assert call(ws=vp((16 << 20) + 8)) == lap5cg.ERR_WORKSPACE
    assert call(ws=None) == lap5cg.ERR_WORKSPACE
    o = lap5cg.default_opts(rr_period=5)
    assert L.cg_solve(8, 8, 8, vp(1 << 20), vp(2 << 20), 1e-8, 10, 0, 0, 1, ws, big, info, ctypes.byref(o),
                      None) == lap5cg.ERR_INVALID_ARG  # residual replacement is a NewCG option
    # option values outside their documented ranges
    for bad in (dict(lane_vec=3), dict(lane_vec=16), dict(lane_vec=-1), dict(reproducible=2), dict(reproducible=-1),
                dict(mg_nu=-1), dict(mg_levels=-2), dict(ring_slots=99), dict(maxit_inner=-1)):
        o = lap5cg.default_opts(**bad)
        assert L.cg_solve(8, 8, 8, vp(1 << 20), vp(2 << 20), 1e-8, 10, 0, 0, 1, ws, big, info, ctypes.byref(o),
                          None) == lap5cg.ERR_INVALID_ARG, bad


def test_product_path_does_not_import_oracle():
    import sys
    import subprocess
    code = ("import sys; import paper_1803_03797_gb300 as m; m.lib(); "
            "assert not any(k == 'oracle' or k.startswith('oracle.') for k in sys.modules), 'oracle imported'")
    subprocess.run([sys.executable, "-c", code], check=True, cwd=ROOT)
    for f in glob.glob(os.path.join(ROOT, "paper_1803_03797_gb300", "**", "*"), recursive=True):
        if f.endswith((".py", ".cu", ".cuh", ".h")):
            assert "oracle" not in open(f).read().lower().replace("oracles", ""), f
