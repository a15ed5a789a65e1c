"""Python front end of the FP64 CPU oracle (``gs_oracle.c``).

TEST INFRASTRUCTURE ONLY: the tests, the smoke check and the CPU-baseline leg
of the benchmark may import this module; the CUDA library and its Python
binding never do.  The oracle shares no code with the CUDA path; both sides
receive the same float32 arrays from the ``synth`` generators.

Every function takes a ``synth.Scene`` / ``synth.Camera`` (or plain numpy
arrays) and returns numpy arrays.  See ``gs_oracle.c`` for the definitions
each step follows (Section II-B, Eq. 1, Algorithm 1, Appendix B).
"""

from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gs_oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build_oracle(force: bool = False) -> str:
    """Compile the oracle with gcc (OpenMP when available).  IEEE semantics:
    no fast-math, no FMA contraction, so x86 and Arm builds agree."""
    if not force and os.path.exists(_LIB_PATH) and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC):
        return _LIB_PATH
    base = ["gcc", "-O2", "-std=c11", "-D_GNU_SOURCE", "-fPIC", "-shared", "-ffp-contract=off",
            "-fno-fast-math", _SRC, "-lm", "-o", _LIB_PATH + ".tmp"]
    try:
        subprocess.run(base[:1] + ["-fopenmp"] + base[1:], check=True, capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True, capture_output=True)
    os.replace(_LIB_PATH + ".tmp", _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build_oracle()
            lib = ctypes.CDLL(_LIB_PATH)
            P = ctypes.c_void_p
            i64, i32, f64 = ctypes.c_int64, ctypes.c_int, ctypes.c_double
            lib.oracle_preprocess.restype = i64
            lib.oracle_preprocess.argtypes = [i64, P, P, P, P, P, i32, P] + [P] * 12
            lib.oracle_num_instances.restype = i64
            lib.oracle_num_instances.argtypes = [i64, P]
            lib.oracle_duplicate_sort.restype = None
            lib.oracle_duplicate_sort.argtypes = [i64, P, P, P, i32, i32, i64, P, P, P]
            lib.oracle_render.restype = None
            lib.oracle_render.argtypes = [i32, i32, i32, i32, P, P, i64, P, P, P, P, P, P, f64, f64, f64, i32] + [P] * 7
            lib.oracle_render_bruteforce.restype = None
            lib.oracle_render_bruteforce.argtypes = [i32, i32, i64, P, P, P, P, P, P, P, P, P, i32] + [P] * 7
            lib.oracle_sh_basis.restype = f64
            lib.oracle_sh_basis.argtypes = [i32, i32, f64, f64, f64]
            lib.oracle_has_openmp.restype = i32
            _lib = lib
    return _lib


class use_library:
    """Context manager that points this module at another build of the
    oracle (the mutation tests load deliberately broken copies)."""

    def __init__(self, path: str):
        self.path = path

    def __enter__(self):
        global _lib
        _load()
        self._saved = _lib
        lib = ctypes.CDLL(self.path)
        for name in ("oracle_preprocess", "oracle_num_instances", "oracle_duplicate_sort", "oracle_render",
                     "oracle_render_bruteforce", "oracle_sh_basis", "oracle_has_openmp"):
            src = getattr(self._saved, name)
            dst = getattr(lib, name)
            dst.restype, dst.argtypes = src.restype, src.argtypes
        _lib = lib
        return self

    def __exit__(self, *exc):
        global _lib
        _lib = self._saved
        return False


def compile_variant(src_text: str, out_path: str) -> str:
    """Compile a modified copy of the oracle source to ``out_path``."""
    c_path = out_path + ".c"
    with open(c_path, "w") as f:
        f.write(src_text)
    subprocess.run(["gcc", "-O1", "-std=c11", "-D_GNU_SOURCE", "-fPIC", "-shared", "-ffp-contract=off", c_path,
                    "-lm", "-o", out_path], check=True, capture_output=True)
    return out_path


def source_text() -> str:
    with open(_SRC) as f:
        return f.read()


def _p(a: np.ndarray):
    assert a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(ctypes.c_void_p)


def camera_record(cam) -> np.ndarray:
    """The oracle's own flat float32 camera record: viewmat (16, row-major),
    fx, fy, cx, cy, width, height, tan_fovx, tan_fovy."""
    rec = np.zeros(24, np.float32)
    rec[:16] = np.asarray(cam.viewmat, np.float32).reshape(16)
    rec[16:24] = [cam.fx, cam.fy, cam.cx, cam.cy, cam.width, cam.height, cam.tan_fovx, cam.tan_fovy]
    return rec


def sh_basis(l: int, m: int, x: float, y: float, z: float) -> float:
    """Real orthonormal SH Y_l^m (Condon-Shortley phase) at unit direction."""
    return _load().oracle_sh_basis(l, m, x, y, z)


def has_openmp() -> bool:
    return bool(_load().oracle_has_openmp())


def preprocess(scene, cam) -> dict:
    """Per-Gaussian projection, colour, depth, radius and tile rectangle."""
    lib = _load()
    n = scene.n
    f32 = lambda a: np.ascontiguousarray(a, np.float32)
    means, ls, q, op, sh = (f32(a) for a in scene.arrays())
    out = dict(
        xy=np.zeros((n, 2)), cov2d=np.zeros((n, 3)), conic=np.zeros((n, 3)), opacity=np.zeros(n),
        rgb=np.zeros((n, 3)), depth=np.zeros(n), depth32=np.zeros(n, np.float32),
        radius=np.zeros(n, np.int32), rect=np.zeros((n, 4), np.int32), tiles=np.zeros(n, np.int32),
        rad_dist=np.zeros(n), edge_dist=np.zeros(n),
    )
    rec = camera_record(cam)
    vis = lib.oracle_preprocess(n, _p(means), _p(ls), _p(q), _p(op), _p(sh), int(scene.sh_degree), _p(rec),
                                *[_p(out[k]) for k in ("xy", "cov2d", "conic", "opacity", "rgb", "depth",
                                                       "depth32", "radius", "rect", "tiles", "rad_dist",
                                                       "edge_dist")])
    out["visible"] = int(vis)
    return out


def duplicate_sort(pre: dict, cam) -> dict:
    """Key duplication, stable sort by (tile << 32 | depth bits), tile ranges."""
    lib = _load()
    n = pre["tiles"].shape[0]
    m = int(lib.oracle_num_instances(n, _p(pre["tiles"])))
    keys = np.zeros(max(m, 1), np.uint64)
    vals = np.zeros(max(m, 1), np.uint32)
    ranges = np.zeros((cam.num_tiles, 2), np.uint32)
    lib.oracle_duplicate_sort(n, _p(pre["rect"]), _p(pre["tiles"]), _p(pre["depth32"]), cam.tiles_x,
                              cam.num_tiles, m, _p(keys), _p(vals), _p(ranges))
    return dict(keys=keys[:m], vals=vals[:m], ranges=ranges, m=m)


_RENDER_KEYS = ("color", "invdepth", "final_T", "n_contrib", "n_eval", "near", "flip_impact")


def _render_outputs(w: int, h: int) -> dict:
    return dict(color=np.zeros((3, h, w)), invdepth=np.zeros((h, w)), final_T=np.zeros((h, w)),
                n_contrib=np.zeros((h, w), np.int32),
                n_eval=np.zeros((h, w), np.int32), near=np.zeros((h, w), np.int32),
                flip_impact=np.zeros((h, w)))


def render(pre: dict, srt: dict, cam, bg=(0.0, 0.0, 0.0), tau_alpha: float = 0.0, tau_T: float = 0.0,
           rows: tuple | None = None, threads: int = 0, pos_eps: float = 0.0) -> dict:
    """Tiled front-to-back compositing of every pixel in ``rows`` (default:
    all).  ``tau_alpha`` / ``tau_T`` set the log-space margin under which a
    threshold decision counts as near; ``pos_eps`` widens it by the effect of
    that relative rounding of each splat's pixel coordinates.  ``near``
    counts a pixel's near decisions; ``flip_impact`` is the largest change of
    a colour channel when one of them is taken the other way and the rest of
    the list is walked again."""
    lib = _load()
    w, h = cam.width, cam.height
    r0, r1 = (0, h) if rows is None else rows
    out = _render_outputs(w, h)
    bgv = np.ascontiguousarray(bg, np.float64)
    vals = np.ascontiguousarray(srt["vals"] if srt["m"] else np.zeros(1, np.uint32))
    n = pre["xy"].shape[0]
    lib.oracle_render(w, h, r0, r1, _p(np.ascontiguousarray(srt["ranges"])), _p(vals), n, _p(pre["xy"]),
                      _p(pre["conic"]), _p(pre["opacity"]), _p(pre["rgb"]), _p(pre["depth"]), _p(bgv), tau_alpha,
                      tau_T, float(pos_eps), int(threads), *[_p(out[k]) for k in _RENDER_KEYS])
    return out


def render_bruteforce(pre: dict, cam, bg=(0.0, 0.0, 0.0), use_rect: bool = True) -> dict:
    """Per-pixel compositing without tile lists (tiny scenes only)."""
    lib = _load()
    w, h = cam.width, cam.height
    out = _render_outputs(w, h)
    bgv = np.ascontiguousarray(bg, np.float64)
    n = pre["xy"].shape[0]
    lib.oracle_render_bruteforce(w, h, n, _p(pre["rect"]), _p(pre["radius"]), _p(pre["depth32"]),
                                 _p(pre["xy"]), _p(pre["conic"]), _p(pre["opacity"]), _p(pre["rgb"]),
                                 _p(pre["depth"]), _p(bgv), int(use_rect), *[_p(out[k]) for k in _RENDER_KEYS])
    return out


def frame(scene, cam, bg=(0.0, 0.0, 0.0), tau_alpha: float = 0.0, tau_T: float = 0.0, threads: int = 0,
          pos_eps: float = 0.0):
    """Whole forward pass: preprocess, duplicate + sort + ranges, render."""
    pre = preprocess(scene, cam)
    srt = duplicate_sort(pre, cam)
    img = render(pre, srt, cam, bg, tau_alpha, tau_T, threads=threads, pos_eps=pos_eps)
    return pre, srt, img
