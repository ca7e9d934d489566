"""The C-ABI library loads and exports every symbol include/ws.h declares; host-side
argument validation (no GPU needed: these calls fail before any CUDA call)."""
import ctypes
import subprocess

import pytest

from paper_2604_00048_b300 import build as wsbuild


@pytest.fixture(scope="module")
def ws():
    wsbuild.build()
    from paper_2604_00048_b300 import ws as mod
    return mod


def test_exports_every_declared_symbol(ws):
    declared = ws.declared_symbols()
    assert {"ws_smooth_batch", "ws_factor", "ws_solve", "ws_solve_adjoint", "ws_workspace_size"} <= set(declared)
    out = subprocess.run(["nm", "-D", "--defined-only", ws.LIB_PATH], capture_output=True, text=True).stdout
    exported = {l.split()[-1] for l in out.splitlines() if l.strip()}
    missing = [s for s in declared if s not in exported]
    assert not missing, missing
    for s in declared:
        getattr(ws.lib(), s)


def test_version(ws):
    assert "sm_103a" in ws.version()


def test_invalid_problems_rejected_before_cuda(ws):
    bad = [dict(d=0), dict(d=5), dict(n_bands=0), dict(T=-1), dict(dtype=7), dict(lam_mode=3)]
    for kw in bad:
        args = dict(T=10, B=1, P=8, d=2, dtype=ws.F32, lam_mode=ws.LAM_PER_DAY)
        args.update({k: v for k, v in kw.items() if k in ("T", "d", "dtype", "lam_mode")})
        pb = ws.make_problem(args["T"], kw.get("n_bands", 1), 8, args["d"], args["dtype"], args["lam_mode"])
        assert ws.workspace_size(pb) == 0
        rc = ws.lib().ws_smooth_batch(ctypes.byref(pb), None, None, None, None, None, None, 0, None, 0, None)
        assert rc == ws.WS_EINVAL
        assert ws.last_error()


def test_null_pointers_and_flags_rejected(ws):
    pb = ws.make_problem(10, 1, 8, 2, ws.F32, ws.LAM_PER_DAY)
    rc = ws.lib().ws_smooth_batch(ctypes.byref(pb), None, None, None, None, None, None, 0, None, 0, None)
    assert rc == ws.WS_EINVAL and "non-NULL" in ws.last_error()
    rc = ws.lib().ws_smooth_batch(ctypes.byref(pb), None, None, None, None, None, None, 0x80, None, 0, None)
    assert rc == ws.WS_EINVAL and "flags" in ws.last_error()
    assert ws.lib().ws_tune_set(9, 0) == ws.WS_EINVAL
    assert ws.lib().ws_tune_set(2, 300) == ws.WS_EINVAL
    assert ws.lib().ws_tune_set(-1, 0) == ws.WS_EINVAL
    assert ws.lib().ws_tune_set(0, 0) == ws.WS_OK


def test_empty_problem_is_a_no_op(ws):
    pb = ws.make_problem(10, 1, 0, 2, ws.F32, ws.LAM_PER_DAY)
    rc = ws.lib().ws_smooth_batch(ctypes.byref(pb), None, None, None, None, None, None, 0, None, 0, None)
    assert rc == ws.WS_OK
