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
    assert ws.lib().ws_tune_set(33, 0) == ws.WS_EINVAL
    assert ws.lib().ws_tune_set(2, 300) == ws.WS_EINVAL
    assert ws.lib().ws_tune_set(-1, 0) == ws.WS_EINVAL
    assert ws.lib().ws_tune_set(0, 0) == ws.WS_OK
    assert ws.lib().ws_tune_checkpoint_group(3) == ws.WS_EINVAL
    assert ws.lib().ws_tune_checkpoint_group(-1) == ws.WS_EINVAL
    assert ws.lib().ws_tune_checkpoint_group(0) == ws.WS_OK


def test_empty_problem_is_a_no_op(ws):
    pb = ws.make_problem(10, 1, 0, 2, ws.F32, ws.LAM_PER_DAY)
    rc = ws.lib().ws_smooth_batch(ctypes.byref(pb), None, None, None, None, None, None, 0, None, 0, None)
    assert rc == ws.WS_OK


def test_gcv_argument_checks(ws):
    pb = ws.make_problem(30, 1, 8, 2, ws.F32, ws.LAM_SCALAR)
    grid = (ctypes.c_float * 3)(1.0, 10.0, 100.0)
    call = ws.lib().ws_gcv_smooth
    assert call(ctypes.byref(pb), None, None, grid, 0, None, None, None, None, 0, None, 0, None) == ws.WS_EINVAL
    assert call(ctypes.byref(pb), None, None, grid, 17, None, None, None, None, 0, None, 0, None) == ws.WS_EINVAL
    bad = (ctypes.c_float * 2)(1.0, -2.0)
    assert call(ctypes.byref(pb), None, None, bad, 2, None, None, None, None, 0, None, 0, None) == ws.WS_EINVAL
    assert "lam_grid" in ws.last_error()
    pb64 = ws.make_problem(30, 1, 8, 2, ws.F64, ws.LAM_SCALAR)
    assert call(ctypes.byref(pb64), None, None, grid, 3, None, None, None, None, 0, None, 0, None) == ws.WS_EUNSUPPORTED
    pb3 = ws.make_problem(30, 3, 8, 2, ws.F32, ws.LAM_SCALAR)
    assert call(ctypes.byref(pb3), None, None, grid, 3, None, None, None, None, 0, None, 0, None) == ws.WS_EUNSUPPORTED


def test_network_argument_checks(ws):
    lib = ws.lib()
    good = ws.TcnBatch(730, 16, *ws.TCN_LOG_LAM)
    n0 = lib.ws_tcn_scratch_size(ctypes.byref(good), 0)
    n1 = lib.ws_tcn_scratch_size(ctypes.byref(good), 1)
    rows = 16 * (730 + ws.TCN_GAP)
    assert n0 >= rows * 8 and n1 >= n0 + rows * 128 * 5  # training keeps 3 activation + 2 gradient arrays
    assert lib.ws_tcn_scratch_size(ctypes.byref(ws.TcnBatch(0, 16, 0.0, 1.0)), 0) == 0
    assert lib.ws_tcn_scratch_size(ctypes.byref(ws.TcnBatch(10, 16, 2.0, 1.0)), 0) == 0
    assert lib.ws_tcn_forward(ctypes.byref(good), None, None, None, None, None, None, None, 0, 0, None) == ws.WS_EINVAL
    fake = ctypes.c_void_p(256)  # never dereferenced: the size check fails first
    assert lib.ws_tcn_forward(ctypes.byref(good), fake, fake, fake, fake, fake, None, fake, 16, 0, None) == ws.WS_ENOMEM_WS
    assert lib.ws_tcn_backward(ctypes.byref(good), None, None, None, None, 0, None) == ws.WS_EINVAL
    assert lib.ws_adam_step(None, None, None, None, 10, 1, 1e-3, 0.9, 0.999, 1e-8, None) == ws.WS_EINVAL
    assert lib.ws_adam_step(fake, fake, fake, fake, 10, 0, 1e-3, 0.9, 0.999, 1e-8, None) == ws.WS_EINVAL
    assert lib.ws_mse_grad(None, None, None, None, 10, 1.0, None) == ws.WS_EINVAL
    assert lib.ws_tcn_conv64(fake, fake, None, None, fake, 10, 5, 0, fake, None) == ws.WS_EINVAL  # forward needs bias
    assert lib.ws_tcn_conv64(fake, fake, None, None, fake, 10, 5, 1, fake, None) == ws.WS_EINVAL  # gradient needs mask
    assert lib.ws_tcn_conv64(fake, fake, fake, fake, fake, 10, 5, 2, fake, None) == ws.WS_EINVAL  # mode


def test_noalloc_and_plan_argument_checks(ws):
    lib = ws.lib()
    assert lib.ws_smooth_batch_noalloc(None, None, None, None, None, None, None, 0, None) == ws.WS_EINVAL
    bad = ws.make_problem(10, 1, 8, 0, ws.F32, ws.LAM_PER_DAY)
    assert lib.ws_smooth_batch_noalloc(ctypes.byref(bad), None, None, None, None, None, None, 0, None) == ws.WS_EINVAL
    h = ctypes.c_void_p()
    assert lib.ws_plan_create(None, ctypes.byref(h), None) == ws.WS_EINVAL
    rg = ws.Ragged(4, None, None, 2, 1, ws.F32, ws.LAM_PER_DAY)
    assert lib.ws_plan_create(ctypes.byref(rg), ctypes.byref(h), None) == ws.WS_EINVAL  # offsets NULL
    rg64 = ws.Ragged(4, 256, None, 2, 1, ws.F64, ws.LAM_PER_DAY)  # rejected before the offsets are read
    assert lib.ws_plan_create(ctypes.byref(rg64), ctypes.byref(h), None) == ws.WS_EUNSUPPORTED
    assert lib.ws_plan_execute(None, None, None, None, None, None, 0, None, 0, None) == ws.WS_EINVAL
    assert lib.ws_plan_workspace_size(None, 0) == 0
    assert lib.ws_plan_info(None, None) == ws.WS_EINVAL


def test_posterior_arguments_rejected_before_cuda(ws):
    """ws_posterior: invalid problem, NULL outputs or inputs, outputs overlapping the inputs
    or each other, all rejected with WS_EINVAL before any CUDA call; P = 0 is a no-op."""
    L = ws.lib()
    pb = ws.make_problem(10, 2, 8, 5, ws.F32, ws.LAM_PER_DAY)
    assert L.ws_posterior(ctypes.byref(pb), *([None] * 8), None, 0, None) == ws.WS_EINVAL
    pb = ws.make_problem(10, 2, 8, 2, ws.F32, ws.LAM_PER_DAY)
    assert L.ws_posterior(ctypes.byref(pb), *([None] * 8), None, 0, None) == ws.WS_EINVAL
    assert "sigma2" in ws.last_error()
    # fake, never dereferenced device addresses: x, w, lam, z at distinct ranges
    T, B, P = 10, 2, 8
    nx, nd = T * B * P * 4, T * P * 4
    base = 1 << 40
    x, w, lam, z = base, base + 4096, base + 8192, base + 12288
    diag, s2, sd = base + 16384, base + 20480, base + 24576
    assert L.ws_posterior(ctypes.byref(pb), x, w, lam, z, None, s2, sd, None, None, 0, None) == ws.WS_EINVAL
    assert "non-NULL" in ws.last_error()
    assert L.ws_posterior(ctypes.byref(pb), x, w, lam, z, x + 64, s2, sd, None, None, 0, None) == ws.WS_EINVAL
    assert "overlap" in ws.last_error()
    assert L.ws_posterior(ctypes.byref(pb), x, w, lam, z, diag, diag + 16, sd, None, None, 0, None) == ws.WS_EINVAL
    assert "overlap" in ws.last_error()
    assert L.ws_posterior(ctypes.byref(pb), x, w, lam, z, diag, s2, z + nx - 4, None, None, 0, None) == ws.WS_EINVAL
    assert nd < 4096 and nx < 4096
    pb0 = ws.make_problem(10, 2, 0, 2, ws.F32, ws.LAM_PER_DAY)
    assert L.ws_posterior(ctypes.byref(pb0), *([None] * 8), None, 0, None) == ws.WS_OK


def test_weight_grad_arguments_rejected_before_cuda(ws):
    """ws_weight_grad: NULL inputs/outputs and overlaps rejected with WS_EINVAL before any
    CUDA call; gx == g (in place) is accepted by the checks; empty problems are no-ops."""
    L = ws.lib()
    T, B, P = 10, 2, 8
    pb = ws.make_problem(T, B, P, 2, ws.F32, ws.LAM_PER_DAY)
    nx, nd = T * B * P * 4, T * P * 4
    base = 1 << 40
    x, w, z, g, gw, gx = base, base + 4096, base + 8192, base + 12288, base + 16384, base + 20480
    assert L.ws_weight_grad(ctypes.byref(pb), None, w, z, g, gx, gw, None) == ws.WS_EINVAL
    assert "non-NULL" in ws.last_error()
    assert L.ws_weight_grad(ctypes.byref(pb), x, w, z, g, gx, None, None) == ws.WS_EINVAL
    assert L.ws_weight_grad(ctypes.byref(pb), x, w, z, g, g + 4, gw, None) == ws.WS_EINVAL
    assert "gx" in ws.last_error()
    assert L.ws_weight_grad(ctypes.byref(pb), x, w, z, g, gx, z + 16, None) == ws.WS_EINVAL
    assert L.ws_weight_grad(ctypes.byref(pb), x, w, z, g, x, gw, None) == ws.WS_EINVAL
    assert nx < 4096 and nd < 4096
    for pb0 in (ws.make_problem(T, B, 0, 2, ws.F32, ws.LAM_PER_DAY), ws.make_problem(0, B, P, 2, ws.F32, ws.LAM_PER_DAY)):
        assert L.ws_weight_grad(ctypes.byref(pb0), None, None, None, None, None, None, None) == ws.WS_OK
    pb = ws.make_problem(T, B, P, 2, ws.F32, ws.LAM_PER_DAY)
    rc = L.ws_solve_adjoint(ctypes.byref(pb), None, None, None, None, None, None, None, 0x40, None, None, 0, None)
    assert rc == ws.WS_EINVAL and "flags" in ws.last_error()


def test_dates_arguments_rejected_before_cuda(ws):
    """ws_smooth_dates / ws_smooth_dates_adjoint: NULL arrays, overlapping outputs and unknown
    flags rejected with WS_EINVAL before any CUDA call; P = 0 is a no-op."""
    L = ws.lib()
    T, B, P = 10, 2, 8
    pb = ws.make_problem(T, B, P, 2, ws.F32, ws.LAM_PER_DAY)
    base = 1 << 40
    t, x, w, lam, z, gz, gx, gl = (base + 4096 * i for i in range(8))
    assert L.ws_smooth_dates(ctypes.byref(pb), None, x, w, lam, z, None, 0, None, 0, None) == ws.WS_EINVAL
    assert "non-NULL" in ws.last_error()
    assert L.ws_smooth_dates(ctypes.byref(pb), t, x, w, lam, x + 8, None, 0, None, 0, None) == ws.WS_EINVAL
    assert "overlap" in ws.last_error()
    assert L.ws_smooth_dates(ctypes.byref(pb), t, x, w, lam, z, None, 0x80, None, 0, None) == ws.WS_EINVAL
    assert "flags" in ws.last_error()
    assert L.ws_smooth_dates_adjoint(ctypes.byref(pb), t, w, lam, z, gz, None, gl, 0, None, None, 0, None) == ws.WS_EINVAL
    assert L.ws_smooth_dates_adjoint(ctypes.byref(pb), t, w, lam, z, gz, gz + 4, gl, 0, None, None, 0, None) == ws.WS_EINVAL
    assert L.ws_smooth_dates_adjoint(ctypes.byref(pb), t, w, lam, z, gz, gx, gx, 0, None, None, 0, None) == ws.WS_EINVAL
    assert L.ws_smooth_dates_adjoint(ctypes.byref(pb), t, w, lam, z, gz, gx, gl, 0x80, None, None, 0, None) == ws.WS_EINVAL
    assert "flags" in ws.last_error()
    pb0 = ws.make_problem(T, B, 0, 2, ws.F32, ws.LAM_PER_DAY)
    assert L.ws_smooth_dates(ctypes.byref(pb0), None, None, None, None, None, None, 0, None, 0, None) == ws.WS_OK
    assert L.ws_smooth_dates_adjoint(ctypes.byref(pb0), *([None] * 7), 0, None, None, 0, None) == ws.WS_OK


def test_posterior_dates_arguments_rejected_before_cuda(ws):
    """ws_posterior_dates: a NULL t (with days and series), and the other checks of
    ws_posterior, before any CUDA call; P = 0 is a no-op."""
    L = ws.lib()
    pb = ws.make_problem(10, 2, 8, 2, ws.F32, ws.LAM_PER_DAY)
    base = 1 << 40
    x, w, lam, z, diag, s2, sd = (base + 4096 * i for i in range(7))
    assert L.ws_posterior_dates(ctypes.byref(pb), None, x, w, lam, z, diag, s2, sd, None, None, 0, None) == ws.WS_EINVAL
    assert "t must be" in ws.last_error()
    t = base + 4096 * 8
    assert L.ws_posterior_dates(ctypes.byref(pb), t, x, w, lam, z, x + 4, s2, sd, None, None, 0, None) == ws.WS_EINVAL
    pb0 = ws.make_problem(10, 2, 0, 2, ws.F32, ws.LAM_PER_DAY)
    assert L.ws_posterior_dates(ctypes.byref(pb0), *([None] * 9), None, 0, None) == ws.WS_OK


def test_gcv_dates_arguments_rejected_before_cuda(ws):
    """ws_gcv_smooth_dates: FP64 or several bands unsupported, a bad grid or NULL arrays
    rejected, before any CUDA call."""
    L = ws.lib()
    arr = (ctypes.c_float * 2)(1.0, 10.0)
    pb = ws.make_problem(10, 1, 8, 2, ws.F64, ws.LAM_SCALAR)
    assert L.ws_gcv_smooth_dates(ctypes.byref(pb), None, None, None, arr, 2, *([None] * 4), 0, None, 0, None) == \
        ws.WS_EUNSUPPORTED
    pb = ws.make_problem(10, 1, 8, 2, ws.F32, ws.LAM_SCALAR)
    assert L.ws_gcv_smooth_dates(ctypes.byref(pb), None, None, None, arr, 0, *([None] * 4), 0, None, 0, None) == \
        ws.WS_EINVAL
    assert L.ws_gcv_smooth_dates(ctypes.byref(pb), None, None, None, arr, 2, *([None] * 4), 0, None, 0, None) == \
        ws.WS_EINVAL
    assert "non-NULL" in ws.last_error()


def test_selftest_wait_arguments_rejected_before_cuda(ws):
    L = ws.lib()
    assert L.ws_selftest_wait(None, 4096, None) == ws.WS_EINVAL
    assert L.ws_selftest_wait(ctypes.c_void_p(1 << 40), 16, None) == ws.WS_EINVAL
    assert L.ws_selftest_wait(ctypes.c_void_p((1 << 40) + 8), 4096, None) == ws.WS_EINVAL
