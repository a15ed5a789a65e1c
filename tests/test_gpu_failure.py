"""Failure detection on the device: a bounded wait that runs out.

gs_sort's radix passes learn earlier blocks' digit counts by decoupled
look-back, waiting on flags that other blocks publish.  If a predecessor
never publishes (it stalled or died), the wait must give up, record a
timeout, and let the call report GS_ERR_TIMEOUT, leaving the context usable.
gs_check_wait_timeout runs that very wait against a predecessor that never
runs (a flag nothing sets) with a short limit; nothing here faults, traps or
hangs the GPU.
"""

import ctypes
import time

import pytest
import torch

import paper_2509_25626_gb300 as gs
from paper_2509_25626_gb300 import _lib as L
from synth import tiny_scene

pytestmark = pytest.mark.gpu


def _workspace():
    nbytes = int(L.lib().gs_sort_workspace_bytes(1, 1, 1))
    ws = torch.zeros(nbytes, dtype=torch.uint8, device="cuda")
    assert ws.data_ptr() % 256 == 0
    return ws, nbytes


def test_lookback_wait_gives_up_and_reports_timeout():
    lib = L.lib()
    ws, nbytes = _workspace()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    P = ctypes.c_void_p
    for limit_ms in (5, 40):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        code = lib.gs_check_wait_timeout(P(ws.data_ptr()), nbytes, limit_ms * 1_000_000, stream)
        dt = time.perf_counter() - t0
        assert code == L.GS_ERR_TIMEOUT, L.strerror(code)
        # gave up after its limit, not at once and not after the default 1 s
        assert limit_ms / 1000.0 <= dt < limit_ms / 1000.0 + 0.5, dt
        # the public status call reads the same header record
        m = ctypes.c_int64(-1)
        assert lib.gs_sort_status(P(ws.data_ptr()), ctypes.byref(m), stream) == L.GS_ERR_TIMEOUT


def test_context_usable_after_a_timeout():
    """After the timed-out wait, the same workspace and stream serve a real
    sort, whose status is clean (each gs_sort clears its header)."""
    lib = L.lib()
    ws, nbytes = _workspace()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    assert lib.gs_check_wait_timeout(ctypes.c_void_p(ws.data_ptr()), nbytes, 2_000_000, stream) == \
        L.GS_ERR_TIMEOUT
    sc, cam = tiny_scene(2000, 3, 96, 64)
    st = gs.SceneTensors.from_scene(sc, "cuda")
    sp = gs.preprocess(st, cam)
    keys, vals, ranges, m, wsp = gs.sort(sp, sc.n, cam, 1 << 16)
    torch.cuda.synchronize()
    assert m > 0
    mm = ctypes.c_int64(-1)
    assert lib.gs_sort_status(ctypes.c_void_p(wsp.data_ptr()), ctypes.byref(mm), stream) == L.GS_OK
    assert mm.value == m
