"""The C ABI library: it loads, exports every entry point include/gs.h
declares, and rejects bad arguments before touching the GPU.  No GPU needed."""

import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    from paper_2509_25626_gb300 import build
    build.build()
    from paper_2509_25626_gb300 import _lib
    return _lib


def declared_functions():
    src = open(os.path.join(ROOT, "include", "gs.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(gs_[a-z_]+)\s*\(", src)))


def test_header_declares_the_entry_points():
    names = declared_functions()
    for n in ("gs_preprocess", "gs_sort", "gs_render", "gs_sort_workspace_bytes", "gs_strerror"):
        assert n in names


def test_library_exports_every_declared_symbol(L):
    out = subprocess.run(["nm", "-D", "--defined-only", L.LIB_PATH], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\s[TW]\s+(gs_\w+)", out))
    missing = [n for n in declared_functions() if n not in exported]
    assert not missing, missing
    lib = L.lib()
    for n in declared_functions():
        assert hasattr(lib, n)


def test_built_for_sm103(L):
    assert L.lib().gs_built_arch() == 103
    assert L.lib().gs_version() >= 1


def test_strerror_texts(L):
    for code in (0, -1, -2, -3, -4, -99):
        assert isinstance(L.strerror(code), str) and L.strerror(code)


def _cam(L, w=64, h=48):
    c = L.GsCamera()
    for i in (0, 5, 10, 15):
        c.viewmat[i] = 1.0
    c.fx = c.fy = 55.0
    c.cx, c.cy = (w - 1) / 2, (h - 1) / 2
    c.width, c.height = w, h
    c.tan_fovx, c.tan_fovy = w / 110.0, h / 110.0
    return c


def test_invalid_arguments_rejected_on_host(L):
    lib = L.lib()
    cam = _cam(L)
    sc = L.GsScene()
    sc.n = 10
    # null device pointers
    assert lib.gs_preprocess(ctypes.byref(sc), ctypes.byref(cam), None, None) == L.GS_ERR_INVALID_ARG
    # misaligned
    sc.means = sc.log_scales = sc.quats = sc.opacity_logits = sc.sh = 16 * 1000 + 4
    assert lib.gs_preprocess(ctypes.byref(sc), ctypes.byref(cam), ctypes.c_void_p(16 * 2000), None) == \
        L.GS_ERR_INVALID_ARG
    sc.sh_degree = 4
    assert lib.gs_preprocess(ctypes.byref(sc), ctypes.byref(cam), None, None) == L.GS_ERR_INVALID_ARG
    bad = _cam(L)
    bad.width = 0
    sc.n = 0
    sc.sh_degree = 3
    assert lib.gs_preprocess(ctypes.byref(sc), ctypes.byref(bad), None, None) == L.GS_ERR_INVALID_ARG
    bad = _cam(L)
    bad.fx = float("nan")
    assert lib.gs_preprocess(ctypes.byref(sc), ctypes.byref(bad), None, None) == L.GS_ERR_INVALID_ARG
    # gs_sort: workspace too small, misaligned, capacity too large
    m = ctypes.c_int64()
    P = ctypes.c_void_p
    assert lib.gs_sort(P(256), 10, ctypes.byref(cam), P(256), P(256), 100, P(256), P(256), 8, ctypes.byref(m),
                       None) == L.GS_ERR_INVALID_ARG
    assert lib.gs_sort(P(256), 10, ctypes.byref(cam), P(256), P(256), 100, P(256), P(260), 1 << 30,
                       ctypes.byref(m), None) == L.GS_ERR_INVALID_ARG
    assert lib.gs_sort(P(256), 10, ctypes.byref(cam), P(256), P(256), 1 << 40, P(256), P(256), 1 << 60,
                       ctypes.byref(m), None) == L.GS_ERR_INVALID_ARG
    assert lib.gs_sort(P(256), -1, ctypes.byref(cam), P(256), P(256), 100, P(256), P(256), 1 << 30,
                       ctypes.byref(m), None) == L.GS_ERR_INVALID_ARG
    # gs_render: null outputs, non-finite background
    bg = (ctypes.c_float * 3)(0, 0, 0)
    assert lib.gs_render(P(256), P(256), P(256), ctypes.byref(cam), bg, None, P(256), P(256), None) == \
        L.GS_ERR_INVALID_ARG
    bg_nan = (ctypes.c_float * 3)(0, float("inf"), 0)
    assert lib.gs_render(P(256), P(256), P(256), ctypes.byref(cam), bg_nan, P(256), P(256), P(256), None) == \
        L.GS_ERR_INVALID_ARG
    assert lib.gs_sort_status(None, ctypes.byref(m), None) == L.GS_ERR_INVALID_ARG
    # gs_check_wait_timeout: null, misaligned or small workspace, limit outside 1 .. 1e9 ns
    ws_bytes = lib.gs_sort_workspace_bytes(1, 1, 1)
    assert lib.gs_check_wait_timeout(None, ws_bytes, 1000, None) == L.GS_ERR_INVALID_ARG
    assert lib.gs_check_wait_timeout(P(256 + 16), ws_bytes, 1000, None) == L.GS_ERR_INVALID_ARG
    assert lib.gs_check_wait_timeout(P(256), ws_bytes - 1, 1000, None) == L.GS_ERR_INVALID_ARG
    assert lib.gs_check_wait_timeout(P(256), ws_bytes, 0, None) == L.GS_ERR_INVALID_ARG
    assert lib.gs_check_wait_timeout(P(256), ws_bytes, 2_000_000_000, None) == L.GS_ERR_INVALID_ARG


def test_workspace_size_monotone(L):
    lib = L.lib()
    a = lib.gs_sort_workspace_bytes(1000, 10_000, 100)
    b = lib.gs_sort_workspace_bytes(2000, 10_000, 100)
    c = lib.gs_sort_workspace_bytes(2000, 20_000, 100)
    assert 0 < a < b < c
    assert lib.gs_sort_workspace_bytes(0, 0, 1) > 0


def test_balance_params_checked_on_host(L):
    """gs_render_batch_balanced rejects bad settings and a short workspace
    before any launch."""
    lib = L.lib()
    P = ctypes.c_void_p
    ok = L.GsBalanceParams(4096, 1024, 4096, 256, 32, 1024)
    need = lib.gs_render_balance_workspace_bytes(ctypes.byref(ok))
    assert need > 256
    no_split = L.GsBalanceParams(4096, 1024, 0, 0, 0, 0)  # chunks unused without a budget
    assert 0 < lib.gs_render_balance_workspace_bytes(ctypes.byref(no_split)) < need
    for bad in (L.GsBalanceParams(-1, 1024, 0, 0, 0, 0), L.GsBalanceParams(4096, 1024, 4096, 256, 0, 1024),
                L.GsBalanceParams(4096, 1024, 4096, 256, 65, 1024), L.GsBalanceParams(4096, 1024, 4096, 256, 32, 0)):
        assert lib.gs_render_balance_workspace_bytes(ctypes.byref(bad)) == 0
        assert lib.gs_render_batch_balanced(P(256), P(256), ctypes.byref(bad), P(256), 1 << 30, 0, None) == \
            L.GS_ERR_INVALID_ARG
    assert lib.gs_render_batch_balanced(P(256), P(256), ctypes.byref(ok), P(256), need - 1, 0, None) == \
        L.GS_ERR_INVALID_ARG
    assert lib.gs_render_batch_balanced(P(256), P(256), ctypes.byref(ok), P(256 + 8), need, 0, None) == \
        L.GS_ERR_INVALID_ARG
    assert lib.gs_render_batch_balanced(P(256), P(256), None, P(256), need, 0, None) == L.GS_ERR_INVALID_ARG


def test_static_sort_scratch_covers_its_limits(L):
    """gs_sort_static's fixed 42 MiB array holds gs_sort's workspace at the
    largest n and m_cap it accepts, for every tile grid (the grid only sets
    how many tile passes are laid out)."""
    lib = L.lib()
    scratch = 42 << 20
    for tiles in (1, 200, 6630, 32400, 65536, 1 << 20, (1 << 31) - 1):
        need = lib.gs_sort_workspace_bytes(L.SORT_STATIC_MAX_GAUSSIANS, L.SORT_STATIC_MAX_INSTANCES, tiles)
        assert 0 < need <= scratch, (tiles, need)


def test_binding_fails_loudly_without_library(tmp_path, monkeypatch):
    from paper_2509_25626_gb300 import _lib
    monkeypatch.setattr(_lib, "LIB_PATH", str(tmp_path / "missing.so"))
    monkeypatch.setattr(_lib, "_lib", None)
    with pytest.raises(RuntimeError):
        _lib.lib()
