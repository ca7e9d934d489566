"""ws_smooth_batch_noalloc (static scratch, no allocation) against ws_smooth_batch with a
caller workspace, on two calls in a row. Collected last; also passes alone in a fresh
process, where its first call does the per-device set-up."""
import pytest
import torch

from paper_2604_00048_b300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ws():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    from paper_2604_00048_b300 import ws as mod
    return mod


def _inputs(recipe, T, B, P, dtype):
    rc = synth.Recipe(**{**synth.RECIPES[recipe].__dict__, "T": T, "n_bands": B})
    out = synth.generate_tile(rc, P, device="cuda", dtype=dtype)
    return out["x"], out["w"], out["lam"]


@pytest.mark.parametrize("refine", [False, True])
@pytest.mark.parametrize("case", [("homo_fp64", 365, 1, 4096, torch.float64),
                                  ("hetero_tile", 300, 3, 1000, torch.float32)])
def test_noalloc_matches_workspace_entry_point(ws, case, refine):
    recipe, T, B, P, dtype = case
    x, w, lam = _inputs(recipe, T, B, P, dtype)
    z_ref, st_ref = ws.smooth(x, w, lam, 2, refine=refine)
    for _ in range(2):  # two calls in a row reuse the same static scratch
        z = torch.full_like(x, float("nan"))
        st = torch.full((P,), 255, dtype=torch.uint8, device="cuda")
        ws.smooth_noalloc(x, w, lam, 2, z=z, status=st, refine=refine)
        torch.cuda.synchronize()
        assert torch.equal(z, z_ref)
        assert torch.equal(st, st_ref)


def test_noalloc_rejects_problem_beyond_static_size(ws):
    """A full 512 x 512 x 3288-day x 10-band tile needs gigabytes of checkpoints: refused
    with ENOMEM_WS before any launch (the tensors are never touched: tiny stand-ins)."""
    T, B, P = 3288, 10, 262144
    x = torch.empty(0, device="cuda")
    pb = ws.make_problem(T, B, P, 2, ws.F32, 0)
    import ctypes
    rc = ws._lib.ws_smooth_batch_noalloc(ctypes.byref(pb), x.data_ptr(), x.data_ptr(), x.data_ptr(),
                                         x.data_ptr(), None, None, 0, None)
    assert rc == ws.WS_ENOMEM_WS
    assert "exceeds the static" in ws.last_error()
