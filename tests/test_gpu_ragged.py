"""Ragged persistent path (ws_plan_*): packed series of different lengths and orders,
against the FP64 banded oracle series by series; CUDA-graph replay and autotuner."""
import numpy as np
import pytest
import torch

from oracle import banded, multiprec
from paper_2604_00048_b300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ws():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    from paper_2604_00048_b300 import ws as mod
    return mod


def _oracle_ragged(out, ids, lam_scalar=False, mp_orders=()):
    """Banded FP64 oracle, one series at a time: returns {id: (z, status)}. Series whose
    order is in mp_orders take z from the 50-digit solve instead: with unsmoothed lambda up
    to 1e5, sparse weights and d = 3, cond(Omega) reaches ~1e13 and FP64 is off by up to
    ~2e-3 (pinned in test_oracle_multiprec.py)."""
    off = out["offsets"].cpu().numpy()
    ords = out["order"].cpu().numpy()
    x, w, lam = (out[k].cpu().double().numpy() for k in ("x", "w", "lam"))
    res = {}
    for i in ids:
        a, b = off[i], off[i + 1]
        T = b - a
        if T == 0:
            res[i] = (np.zeros(0), 0)
            continue
        li = lam[i:i + 1] if lam_scalar else lam[a:b, None]
        z, st = banded.smooth_tile(x[a:b, None, None], w[a:b, None], li, int(ords[i]))
        z = z[:, 0, 0]
        if int(ords[i]) in mp_orders and st[0] == 0:
            z = multiprec.smooth_mp(x[a:b], w[a:b], float(li[0]) if lam_scalar else li[:, 0], int(ords[i]))
        res[i] = (z, int(st[0]))
    return res


def _check(out, z, st, ids, tol=1e-4, lam_scalar=False, mp_orders=()):
    ref = _oracle_ragged(out, ids, lam_scalar, mp_orders)
    off = out["offsets"].cpu().numpy()
    zc = z.cpu().double().numpy()
    stc = st.cpu().numpy()
    worst = 0.0
    for i in ids:
        zr, sr = ref[i]
        assert stc[i] == sr, (i, stc[i], sr)
        if sr == 0 and zr.size:
            zg = zc[off[i]:off[i + 1]]
            worst = max(worst, np.max(np.abs(zg - zr)) / max(np.max(np.abs(zr)), 1e-6))
    assert worst <= tol, worst


@pytest.mark.parametrize("graph", [False, True])
def test_ragged_mixed_lengths_and_orders(ws, graph):
    rc = synth.Recipe(**{**synth.RECIPES["ragged"].__dict__, "p_valid": 1.0, "revisit": 1, "lam_log10": (0.0, 3.0)})
    out = synth.generate_ragged(rc, 700, device="cuda", t_range=(0, 300), orders=(1, 2, 3, 4))
    plan = ws.RaggedPlan(out["offsets"], out["order"])
    z, st = plan.execute(out["x"], out["w"], out["lam"], graph=graph)
    z2, st2 = plan.execute(out["x"], out["w"], out["lam"], graph=graph)
    ws.sync_status()
    assert torch.equal(z, z2) and torch.equal(st, st2)
    _check(out, z, st, range(700))


@pytest.mark.parametrize("graph", [False, True])
def test_ragged_sparse_weights_refined(ws, graph):
    """The ragged recipe's own weights (5-day revisit, p = 0.4, unsmoothed lambda up to 1e5)
    at lengths 120..600: one refinement step."""
    rc = synth.RECIPES["ragged"]
    out = synth.generate_ragged(rc, 500, device="cuda", t_range=(120, 600))
    plan = ws.RaggedPlan(out["offsets"], out["order"])
    z, st = plan.execute(out["x"], out["w"], out["lam"], refine=True, graph=graph)
    z2, _ = plan.execute(out["x"], out["w"], out["lam"], refine=True, graph=graph)
    ws.sync_status()
    assert torch.equal(z, z2)
    # d = 3 with unsmoothed lambda reaches cond(Omega) ~ 1e13: some series need the double-float re-solve
    assert plan.info()["hp_series"] > 0
    _check(out, z, st, range(500), tol=1e-4, mp_orders=(3,))


def test_ragged_refine_well_posed_stays_fp32(ws):
    """Daily weights and lambda <= 1e3: every series settles in FP32, none is re-solved."""
    rc = synth.Recipe(**{**synth.RECIPES["ragged"].__dict__, "p_valid": 1.0, "revisit": 1, "lam_log10": (0.0, 3.0)})
    out = synth.generate_ragged(rc, 300, device="cuda", t_range=(1, 400), orders=(1, 2, 3, 4))
    plan = ws.RaggedPlan(out["offsets"], out["order"])
    z, st = plan.execute(out["x"], out["w"], out["lam"], refine=True)
    ws.sync_status()
    assert plan.info()["hp_series"] == 0
    _check(out, z, st, range(300), tol=1e-5)


def test_ragged_autotune_decides_tiles(ws):
    """With tiles and the autotuner both requested, the plan times the length-class tiles
    against the best per-lane configuration and keeps the faster; the solution is the
    same either way."""
    rc = synth.Recipe(**{**synth.RECIPES["ragged"].__dict__, "p_valid": 1.0, "revisit": 1, "lam_log10": (0.0, 3.0)})
    out = synth.generate_ragged(rc, 600, device="cuda", t_range=(64, 400), orders=(1, 2, 3))
    plan = ws.RaggedPlan(out["offsets"], out["order"])
    z, st = plan.execute(out["x"], out["w"], out["lam"], autotune=True, tiles=True)
    info = plan.info()
    assert info["tuned"] == 1 and info["tiles"] in (0, 1)
    z2, _ = plan.execute(out["x"], out["w"], out["lam"], tiles=True)
    ws.sync_status()
    assert torch.equal(z, z2)
    _check(out, z, st, range(600))


def test_ragged_graph_updates_arguments_and_autotune(ws):
    rc = synth.Recipe(**{**synth.RECIPES["ragged"].__dict__, "p_valid": 1.0, "revisit": 1, "lam_log10": (0.0, 3.0)})
    out = synth.generate_ragged(rc, 300, device="cuda", t_range=(50, 400))
    plan = ws.RaggedPlan(out["offsets"], out["order"])
    z1, _ = plan.execute(out["x"], out["w"], out["lam"], autotune=True, graph=True)
    x2 = out["x"] * 2.0 + 1.0
    z2, _ = plan.execute(x2, out["w"], out["lam"], autotune=True, graph=True)
    z3, _ = plan.execute(x2, out["w"], out["lam"])
    ws.sync_status()
    info = plan.info()
    assert info["tuned"] == 1 and info["graph"] == 1
    assert torch.allclose(z2, z3, rtol=0, atol=0)
    assert not torch.allclose(z1, z2)


def test_ragged_status_and_scalar_lambda(ws):
    rc = synth.Recipe(**{**synth.RECIPES["ragged"].__dict__, "p_valid": 1.0, "revisit": 1})
    out = synth.generate_ragged(rc, 64, device="cuda", t_range=(0, 40), orders=(2,))
    w = out["w"].clone()
    off = out["offsets"].cpu().numpy()
    w[int(off[3]):int(off[4])] = 0.0                  # no weights: not PD (if T >= 1)
    lam = torch.full((64,), 50.0, device="cuda")
    lam[5] = -1.0                                     # invalid scalar lambda
    plan = ws.RaggedPlan(out["offsets"], out["order"], lam_scalar=True)
    z, st = plan.execute(out["x"], w, lam)
    ws.sync_status()
    stc = st.cpu().numpy()
    if off[4] > off[3]:
        assert stc[3] == 1
    if off[6] - off[5] > 2:
        assert stc[5] == 3
    out2 = dict(out)
    out2["w"], out2["lam"] = w, lam
    ids = [i for i in range(64) if i not in (3, 5)]
    _check(out2, z, st, ids, lam_scalar=True)


@pytest.mark.parametrize("tiles", [False, True])
def test_ragged_nonfinite_refined(ws, tiles):
    """A NaN observation on a weighted day: with refinement the series keeps its non-finite
    status (its corrections never settle and it goes on to the double-float re-solve, which
    meets the same NaN), and every other series still matches the oracle (lengths 64..300:
    with tiles they go through the length classes and their tile refinement step)."""
    rc = synth.Recipe(**{**synth.RECIPES["ragged"].__dict__, "p_valid": 1.0, "revisit": 1, "lam_log10": (0.0, 3.0)})
    out = synth.generate_ragged(rc, 200, device="cuda", t_range=(64, 300), orders=(1, 2, 3))
    off = out["offsets"].cpu().numpy()
    x = out["x"].clone()
    x[int(off[7]) + 10] = float("nan")
    out2 = dict(out)
    out2["x"] = x
    plan = ws.RaggedPlan(out["offsets"], out["order"])
    z, st = plan.execute(x, out["w"], out["lam"], refine=True, tiles=tiles)
    ws.sync_status()
    stc = st.cpu().numpy()
    assert stc[7] == ws.SERIES_NONFINITE
    ids = [i for i in range(200) if i != 7]
    assert np.all(stc[ids] == 0)
    _check(out2, z, st, ids, tol=1e-4)


@pytest.mark.parametrize("tiles", [False, True])
def test_ragged_full_size_sampled(ws, tiles):
    """1,048,576 series, T ~ U{120..3288}, d in {1,2,3} in equal thirds, per-day
    lambda = 10^U[0,5]: autotuned, graph-replayed, refined (FP32 steps, double-float
    re-solve); with tiles the series of 64 days or more are solved and take their first
    refinement step on the length-class tiles (the configuration the bench times). 1024
    sampled series: those of order 1 and 2 against the banded FP64 oracle, the first 64 of
    order 3 against the 50-digit solve (FP64 is not a reference there)."""
    rc = synth.RECIPES["ragged"]
    out = synth.generate_ragged(rc, 1 << 20, device="cuda")
    plan = ws.RaggedPlan(out["offsets"], out["order"])
    z, st = plan.execute(out["x"], out["w"], out["lam"], autotune=not tiles, graph=True, refine=True, tiles=tiles)
    ws.sync_status()
    ids = np.random.default_rng(11).choice(1 << 20, 1024, replace=False)
    ords = out["order"].cpu().numpy()
    _check(out, z, st, [i for i in ids if ords[i] < 3], tol=1e-4)
    _check(out, z, st, [i for i in ids if ords[i] == 3][:64], tol=1e-4, mp_orders=(3,))


def test_ragged_scalar_lambda_refined(ws):
    """One lambda per series (Eq. 2), sparse weights, orders 1..3, with refinement."""
    rc = synth.Recipe(**{**synth.RECIPES["ragged"].__dict__, "lam_kind": "scalar", "lam_log10": (0.0, 5.0)})
    out = synth.generate_ragged(rc, 300, device="cuda", t_range=(60, 400))
    lam = out["lam"]
    off = out["offsets"]
    lam_s = lam[off[:-1].clamp(max=lam.numel() - 1)].contiguous()  # per series: its first day's value
    plan = ws.RaggedPlan(out["offsets"], out["order"], lam_scalar=True)
    z, st = plan.execute(out["x"], out["w"], lam_s, refine=True)
    ws.sync_status()
    out2 = dict(out)
    out2["lam"] = lam_s
    _check(out2, z, st, range(300), tol=1e-4, lam_scalar=True, mp_orders=(3,))


@pytest.mark.parametrize("graph", [False, True])
def test_ragged_tiles_mixed_lengths(ws, graph):
    """WS_PLAN_TILES: series of 64 days or more go through length-class tiles (zero-weight
    padding to a multiple of 32 days), shorter ones through the per-lane kernel; both agree
    with the oracle, repeated executions (graph replay with new buffers) give the same z."""
    rc = synth.Recipe(**{**synth.RECIPES["ragged"].__dict__, "p_valid": 1.0, "revisit": 1, "lam_log10": (0.0, 3.0)})
    out = synth.generate_ragged(rc, 900, device="cuda", t_range=(0, 700), orders=(1, 2, 3, 4))
    plan = ws.RaggedPlan(out["offsets"], out["order"])
    z, st = plan.execute(out["x"], out["w"], out["lam"], graph=graph, tiles=True)
    z2, st2 = plan.execute(out["x"].clone(), out["w"].clone(), out["lam"].clone(), graph=graph, tiles=True)
    ws.sync_status()
    assert torch.equal(z, z2) and torch.equal(st, st2)
    _check(out, z, st, range(900), tol=1e-4)


def test_ragged_tiles_sparse_refined(ws):
    """The ragged recipe's sparse weights and unsmoothed lambda with tiles and refinement."""
    rc = synth.RECIPES["ragged"]
    out = synth.generate_ragged(rc, 400, device="cuda", t_range=(40, 600))
    plan = ws.RaggedPlan(out["offsets"], out["order"])
    z, st = plan.execute(out["x"], out["w"], out["lam"], refine=True, graph=True, tiles=True)
    ws.sync_status()
    _check(out, z, st, range(400), tol=1e-4, mp_orders=(3,))


def test_ragged_execute_captured_in_callers_graph(ws):
    """The call path allocates nothing and never synchronises: ws_plan_execute with
    WS_PLAN_TILES | WS_PLAN_REFINE on a caller-owned workspace is captured into the caller's
    CUDA graph (torch's capture, which rejects allocation and synchronising calls), and a
    replay reproduces the eager result exactly (each series' arithmetic does not depend on
    which item or launch order runs it)."""
    rc = synth.RECIPES["ragged"]
    out = synth.generate_ragged(rc, 700, device="cuda", t_range=(40, 900))
    plan = ws.RaggedPlan(out["offsets"], out["order"])
    need = plan.workspace_size(refine=True, tiles=True)
    assert need > 0 and need >= plan.workspace_size(tiles=True) and need >= plan.workspace_size(refine=True)
    wsb = torch.zeros(need, dtype=torch.uint8, device="cuda")
    z0, st0 = plan.execute(out["x"], out["w"], out["lam"], refine=True, tiles=True, workspace_buf=wsb)
    torch.cuda.synchronize()
    z = torch.full_like(out["x"], float("nan"))
    st = torch.full_like(st0, 255)
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    g = torch.cuda.CUDAGraph()
    with torch.cuda.stream(s):
        # thread-local capture: this thread's allocating or synchronising calls fail it
        with torch.cuda.graph(g, stream=s, capture_error_mode="thread_local"):
            plan.execute(out["x"], out["w"], out["lam"], z=z, status=st, refine=True, tiles=True,
                         workspace_buf=wsb, stream=s)
    g.replay()
    torch.cuda.synchronize()
    assert torch.equal(z, z0) and torch.equal(st, st0)
    _check(out, z, st, range(700), tol=1e-4, mp_orders=(3,))
    # a workspace one byte short is rejected before any launch
    flags = ws.PLAN_REFINE | ws.PLAN_TILES
    rc = ws.lib().ws_plan_execute(plan._h, out["x"].data_ptr(), out["w"].data_ptr(), out["lam"].data_ptr(),
                                  z.data_ptr(), st.data_ptr(), flags, wsb.data_ptr(), need - 1, None)
    assert rc == ws.WS_ENOMEM_WS
