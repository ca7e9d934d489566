"""The bounded device-side waits give up cleanly: a kernel waits on an mbarrier that no
thread arrives at (ws_selftest_wait); after the wait limit it records the timeout, the host
reads WS_ETIMEOUT through ws_sync_status, the error word is cleared, and the same context
then smooths correctly. No fault, trap or unbounded wait is involved."""
import ctypes

import numpy as np
import pytest
import torch

from oracle import dense
from tests.gpu_util import rel_err_per_series, tile_inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ws():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    from paper_2604_00048_b300 import ws as mod
    return mod


def test_wait_gives_up_and_context_stays_usable(ws):
    L = ws.lib()
    wsp = torch.zeros(4096, dtype=torch.uint8, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    assert L.ws_sync_status(ws._ptr(wsp), wsp.numel(), ctypes.c_void_p(stream)) == ws.WS_OK
    assert L.ws_selftest_wait(ws._ptr(wsp), wsp.numel(), ctypes.c_void_p(stream)) == ws.WS_OK
    assert L.ws_sync_status(ws._ptr(wsp), wsp.numel(), ctypes.c_void_p(stream)) == ws.WS_ETIMEOUT
    assert "gave up" in ws.last_error()
    assert L.ws_sync_status(ws._ptr(wsp), wsp.numel(), ctypes.c_void_p(stream)) == ws.WS_OK  # cleared
    rc, g, c = tile_inputs("layer", 130, T=60, B=2, revisit=1, p_valid=0.6)
    z, st = ws.smooth(g["x"], g["w"], g["lam"], 2, refine=True)
    ws.sync_status()
    zr, ok = dense.smooth_tile(c["x"], c["w"], c["lam"], 2)
    assert np.array_equal(st.cpu().numpy() == 0, ok)
    assert rel_err_per_series(z.cpu().numpy()[:, :, ok], zr[:, :, ok]) <= 1e-4
