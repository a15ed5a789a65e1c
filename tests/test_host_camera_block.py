"""The kernels' camera block (gs_camera_block), checked on the CPU: it holds
the first three rows of the world-to-camera matrix, the intrinsics, the
tile grid and the camera centre -R^T t formed in double; the server's
block buffers have room for it; invalid cameras are rejected.  No GPU."""

import ctypes
import math

import numpy as np
import pytest

from synth import orbit_camera, pinhole_camera

FIELDS = [("V", ctypes.c_float * 12), ("fx", ctypes.c_float), ("fy", ctypes.c_float), ("cx", ctypes.c_float),
          ("cy", ctypes.c_float), ("tan_fovx", ctypes.c_float), ("tan_fovy", ctypes.c_float),
          ("campos", ctypes.c_float * 3), ("width", ctypes.c_int), ("height", ctypes.c_int),
          ("tiles_x", ctypes.c_int), ("tiles_y", ctypes.c_int)]


class Block(ctypes.Structure):
    _fields_ = FIELDS


@pytest.fixture(scope="module")
def lib():
    from paper_2509_25626_gb300 import build
    build.build()
    from paper_2509_25626_gb300 import _lib
    return _lib


def block_of(lib, cam):
    from paper_2509_25626_gb300.api import camera_struct
    assert lib.lib().gs_camera_block_bytes() == ctypes.sizeof(Block)
    b = Block()
    assert lib.lib().gs_camera_block(ctypes.byref(camera_struct(cam)), ctypes.byref(b)) == 0
    return b


@pytest.mark.parametrize("k", [0, 3, 7, 13])
def test_camera_block_fields(lib, k):
    cam = orbit_camera(k, 20, 4.0, 1237, 822)
    b = block_of(lib, cam)
    vm = np.asarray(cam.viewmat, np.float32).reshape(4, 4)
    assert np.array_equal(np.array(b.V, np.float32), vm[:3].reshape(12))
    assert (b.fx, b.fy, b.cx, b.cy) == tuple(np.float32(v) for v in (cam.fx, cam.fy, cam.cx, cam.cy))
    assert (b.tan_fovx, b.tan_fovy) == (np.float32(cam.tan_fovx), np.float32(cam.tan_fovy))
    assert (b.width, b.height, b.tiles_x, b.tiles_y) == (1237, 822, 78, 52)
    # the camera centre: -R^T t in double, rounded once
    R, t = vm[:3, :3].astype(np.float64), vm[:3, 3].astype(np.float64)
    centre = np.float32(-(R.T @ t))
    assert np.array_equal(np.array(b.campos, np.float32), centre)
    phi = 2.0 * math.pi * k / 20
    assert np.allclose(b.campos, [4.0 * math.sin(phi), 0.0, -4.0 * math.cos(phi)], atol=1e-5)


def test_camera_block_fits_the_server_buffers(lib):
    from paper_2509_25626_gb300.serve import CAM_BLOCK_BYTES
    assert lib.lib().gs_camera_block_bytes() <= CAM_BLOCK_BYTES and CAM_BLOCK_BYTES % 16 == 0


def test_camera_block_rejects_invalid_cameras(lib):
    from paper_2509_25626_gb300.api import camera_struct
    b = Block()
    for w, h in ((0, 10), (10, 0), (-5, 5)):
        cam = pinhole_camera(16, 16)
        c = camera_struct(cam)
        c.width, c.height = w, h
        assert lib.lib().gs_camera_block(ctypes.byref(c), ctypes.byref(b)) == lib.GS_ERR_INVALID_ARG
    assert lib.lib().gs_camera_block(ctypes.byref(camera_struct(pinhole_camera(16, 16))), None) == \
        lib.GS_ERR_INVALID_ARG
