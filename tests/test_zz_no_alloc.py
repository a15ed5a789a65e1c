"""gs_sort_static, the no-allocation variant of gs_sort, checked against gs_sort.

Some callers cannot allocate device memory: a plugin handed only its input
and output buffers, code running inside another framework's memory pool, a
service that reserves all device memory when it starts.  gs_sort_static
serves them by taking its scratch from a fixed array inside the library.
Its sorted keys, values and tile ranges must equal gs_sort's bit for bit
(integer outputs: exact), and must keep doing so call after call, because
every call reuses the same array.  This file is collected last so that a
failure here never hides the rest of the suite.
"""

import ctypes

import pytest
import torch

import paper_2509_25626_gb300 as gs
from paper_2509_25626_gb300 import _lib as L
from synth import clustered_scene, orbit_camera, tiny_scene

pytestmark = pytest.mark.gpu


def _sort_static_through_c_abi(splats, n, cam, m_cap):
    """Calls gs_sort_static through the C ABI; outputs start as garbage."""
    dev = splats.device
    keys = torch.full((max(m_cap, 1),), -7, dtype=torch.int64, device=dev)
    vals = torch.full((max(m_cap, 1),), -7, dtype=torch.int32, device=dev)
    ranges = torch.full((gs.num_tiles(cam), 2), -7, dtype=torch.int32, device=dev)
    m = ctypes.c_int64(-1)
    cam_c = gs.camera_struct(cam)
    P = ctypes.c_void_p
    code = L.lib().gs_sort_static(P(splats.data_ptr()), int(n), ctypes.byref(cam_c), P(keys.data_ptr()),
                                  P(vals.data_ptr()), int(m_cap), P(ranges.data_ptr()), ctypes.byref(m),
                                  P(torch.cuda.current_stream().cuda_stream))
    torch.cuda.synchronize()
    return code, keys, vals, ranges, int(m.value)


def test_sort_static_equals_sort_on_consecutive_calls():
    big = clustered_scene(200_000, seed=4)
    small, small_cam = tiny_scene(5000, 9, 200, 150, log_scale=(-3.0, 0.7))
    cases = [(big, orbit_camera(2, 20, 4.0, 640, 480)), (small, small_cam)]  # large, then smaller
    for scene, cam in cases:
        st = gs.SceneTensors.from_scene(scene, "cuda")
        sp = gs.preprocess(st, cam)
        keys_r, vals_r, ranges_r, m_ref, _ = gs.sort(sp, scene.n, cam, L.SORT_STATIC_MAX_INSTANCES)
        torch.cuda.synchronize()
        assert 0 < m_ref <= L.SORT_STATIC_MAX_INSTANCES
        m_cap = m_ref + 1000
        code, keys_s, vals_s, ranges_s, m_s = _sort_static_through_c_abi(sp, scene.n, cam, m_cap)
        assert code == L.GS_OK, L.strerror(code)
        assert m_s == m_ref
        assert torch.equal(keys_s[:m_ref], keys_r[:m_ref])
        assert torch.equal(vals_s[:m_ref], vals_r[:m_ref])
        assert torch.equal(ranges_s, ranges_r)


def test_sort_static_at_its_documented_limits():
    """n = GS_SORT_STATIC_MAX_GAUSSIANS and m_cap = GS_SORT_STATIC_MAX_INSTANCES
    on a 3840x2160 image (240 x 135 tiles, three tile passes laid out): the
    largest call the header accepts must run and equal gs_sort, and a small
    call right after it must still be exact in the reused array."""
    big, big_cam = tiny_scene(L.SORT_STATIC_MAX_GAUSSIANS, 21, 3840, 2160, log_scale=(-6.5, 0.4))
    small, small_cam = tiny_scene(3000, 8, 120, 90, log_scale=(-3.0, 0.7))
    for scene, cam, m_cap in ((big, big_cam, L.SORT_STATIC_MAX_INSTANCES), (small, small_cam, None)):
        st = gs.SceneTensors.from_scene(scene, "cuda")
        sp = gs.preprocess(st, cam)
        keys_r, vals_r, ranges_r, m_ref, _ = gs.sort(sp, scene.n, cam, L.SORT_STATIC_MAX_INSTANCES)
        torch.cuda.synchronize()
        assert 0 < m_ref <= L.SORT_STATIC_MAX_INSTANCES
        code, keys_s, vals_s, ranges_s, m_s = _sort_static_through_c_abi(sp, scene.n, cam,
                                                                         m_cap if m_cap else m_ref)
        assert code == L.GS_OK, L.strerror(code)
        assert m_s == m_ref
        assert torch.equal(keys_s[:m_ref], keys_r[:m_ref])
        assert torch.equal(vals_s[:m_ref], vals_r[:m_ref])
        assert torch.equal(ranges_s, ranges_r)


def test_sort_static_rejects_sizes_beyond_its_scratch():
    cam = gs.camera_struct(orbit_camera(0, 20, 4.0, 64, 48))
    P = ctypes.c_void_p
    m = ctypes.c_int64(-1)
    lib = L.lib()
    assert lib.gs_sort_static(P(256), L.SORT_STATIC_MAX_GAUSSIANS + 1, ctypes.byref(cam), P(256), P(256), 1000,
                              P(256), ctypes.byref(m), None) == L.GS_ERR_TOO_LARGE
    assert lib.gs_sort_static(P(256), 1000, ctypes.byref(cam), P(256), P(256), L.SORT_STATIC_MAX_INSTANCES + 1,
                              P(256), ctypes.byref(m), None) == L.GS_ERR_TOO_LARGE
    assert "scratch" in L.strerror(L.GS_ERR_TOO_LARGE)
