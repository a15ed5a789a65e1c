"""Thin torch-facing binding of the gs_* C ABI.

Argument marshalling only: every step of the hot path runs in libgs.so.
PyTorch supplies device memory and the current CUDA stream.  Tensors are
passed as raw pointers; dtypes and shapes follow include/gs.h:

    splats   float32 [n, 16]    one 64-byte gs_splat record per Gaussian
    keys     int64   [m_cap]    (tile << 32 | depth bits), sorted
    vals     int32   [m_cap]    Gaussian ids (uint32 bit patterns)
    ranges   int32   [T, 2]     per-tile [start, end)
    image    float32 [3, H, W], final_T float32 [H, W], n_contrib int32 [H, W]
"""

from __future__ import annotations

import ctypes
from dataclasses import dataclass

import numpy as np
import torch

from . import _lib as L


def camera_struct(cam) -> L.GsCamera:
    """gs_camera from any object with viewmat, fx, fy, cx, cy, width, height,
    tan_fovx, tan_fovy attributes."""
    c = L.GsCamera()
    vm = np.ascontiguousarray(np.asarray(cam.viewmat, np.float32).reshape(16))
    ctypes.memmove(c.viewmat, vm.ctypes.data, 64)
    c.fx, c.fy, c.cx, c.cy = float(cam.fx), float(cam.fy), float(cam.cx), float(cam.cy)
    c.width, c.height = int(cam.width), int(cam.height)
    c.tan_fovx, c.tan_fovy = float(cam.tan_fovx), float(cam.tan_fovy)
    return c


def num_tiles(cam) -> int:
    return ((int(cam.width) + 15) // 16) * ((int(cam.height) + 15) // 16)


def _stream(stream=None) -> ctypes.c_void_p:
    s = torch.cuda.current_stream() if stream is None else stream
    return ctypes.c_void_p(int(s.cuda_stream))


def _ptr(t: torch.Tensor | None) -> ctypes.c_void_p:
    return ctypes.c_void_p(0 if t is None else int(t.data_ptr()))


def _check_tensor(t: torch.Tensor, dtype, name: str):
    if not t.is_cuda or t.dtype != dtype or not t.is_contiguous():
        raise ValueError(f"{name}: expected a contiguous CUDA {dtype} tensor, got {t.dtype} on {t.device}")


@dataclass
class SceneTensors:
    means: torch.Tensor
    log_scales: torch.Tensor
    quats: torch.Tensor
    opacity_logits: torch.Tensor
    sh: torch.Tensor
    sh_degree: int = 3

    @property
    def n(self) -> int:
        return int(self.means.shape[0])

    @classmethod
    def from_arrays(cls, means, log_scales, quats, opacity_logits, sh, sh_degree=3, device="cuda"):
        f = lambda a: torch.as_tensor(np.ascontiguousarray(a, np.float32)).to(device).contiguous()
        return cls(f(means), f(log_scales), f(quats), f(opacity_logits), f(sh), int(sh_degree))

    @classmethod
    def from_scene(cls, scene, device="cuda"):
        return cls.from_arrays(scene.means, scene.log_scales, scene.quats, scene.opacity_logits, scene.sh,
                               scene.sh_degree, device)

    def struct(self) -> L.GsScene:
        for name in ("means", "log_scales", "quats", "opacity_logits", "sh"):
            _check_tensor(getattr(self, name), torch.float32, name)
        s = L.GsScene()
        s.means, s.log_scales, s.quats = self.means.data_ptr(), self.log_scales.data_ptr(), self.quats.data_ptr()
        s.opacity_logits, s.sh = self.opacity_logits.data_ptr(), self.sh.data_ptr()
        s.n, s.sh_degree = self.n, int(self.sh_degree)
        return s


def splat_buffer(n: int, device="cuda") -> torch.Tensor:
    """A splat buffer for n Gaussians (gs_splat_buffer_bytes): float32 rows of
    16, the first n rows the records, then the dense sort inputs (4 per row)."""
    n = max(int(n), 1)
    return torch.empty((n + (n + 3) // 4, 16), dtype=torch.float32, device=device)


def preprocess(scene: SceneTensors, cam, splats: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    """gs_preprocess: returns the splat buffer (float32 rows of 16; rows
    [0, n) are the records)."""
    n = scene.n
    if splats is None:
        splats = splat_buffer(n, scene.means.device)
    _check_tensor(splats, torch.float32, "splats")
    c = camera_struct(cam)
    L.check(L.lib().gs_preprocess(ctypes.byref(scene.struct()), ctypes.byref(c), _ptr(splats), _stream(stream)),
            "gs_preprocess")
    return splats


def sort_workspace_bytes(n: int, m_cap: int, tiles: int) -> int:
    return int(L.lib().gs_sort_workspace_bytes(int(n), int(m_cap), int(tiles)))


def sort(splats: torch.Tensor, n: int, cam, m_cap: int, keys=None, vals=None, ranges=None, workspace=None,
         count: bool = True, stream=None):
    """gs_sort.  With count=True the call synchronises once and returns M
    (raising GsError(GS_ERR_CAPACITY) if M > m_cap); otherwise M stays on the
    device and the return value's m is None."""
    dev = splats.device
    T = num_tiles(cam)
    if keys is None:
        keys = torch.empty(max(m_cap, 1), dtype=torch.int64, device=dev)
    if vals is None:
        vals = torch.empty(max(m_cap, 1), dtype=torch.int32, device=dev)
    if ranges is None:
        ranges = torch.empty((T, 2), dtype=torch.int32, device=dev)
    need = sort_workspace_bytes(n, m_cap, T)
    if workspace is None:
        workspace = torch.empty(need, dtype=torch.uint8, device=dev)
    for t, dt, nm in ((keys, torch.int64, "keys"), (vals, torch.int32, "vals"), (ranges, torch.int32, "ranges"),
                      (workspace, torch.uint8, "workspace")):
        _check_tensor(t, dt, nm)
    c = camera_struct(cam)
    m = ctypes.c_int64(-1)
    code = L.lib().gs_sort(_ptr(splats), int(n), ctypes.byref(c), _ptr(keys), _ptr(vals), int(m_cap), _ptr(ranges),
                           _ptr(workspace), workspace.numel(), ctypes.byref(m) if count else None, _stream(stream))
    if code == L.GS_ERR_CAPACITY:
        err = L.GsError(code, "gs_sort")
        err.m = int(m.value)
        raise err
    L.check(code, "gs_sort")
    return keys, vals, ranges, (int(m.value) if count else None), workspace


def sort_static(splats: torch.Tensor, n: int, cam, m_cap: int, keys=None, vals=None, ranges=None,
                count: bool = True, stream=None):
    """gs_sort_static: gs_sort with the library's fixed scratch instead of a
    workspace, for callers that cannot allocate device memory (the keys,
    values and ranges outputs are still the caller's)."""
    dev = splats.device
    T = num_tiles(cam)
    if keys is None:
        keys = torch.empty(max(m_cap, 1), dtype=torch.int64, device=dev)
    if vals is None:
        vals = torch.empty(max(m_cap, 1), dtype=torch.int32, device=dev)
    if ranges is None:
        ranges = torch.empty((T, 2), dtype=torch.int32, device=dev)
    for t, dt, nm in ((keys, torch.int64, "keys"), (vals, torch.int32, "vals"), (ranges, torch.int32, "ranges")):
        _check_tensor(t, dt, nm)
    c = camera_struct(cam)
    m = ctypes.c_int64(-1)
    code = L.lib().gs_sort_static(_ptr(splats), int(n), ctypes.byref(c), _ptr(keys), _ptr(vals), int(m_cap),
                                  _ptr(ranges), ctypes.byref(m) if count else None, _stream(stream))
    L.check(code, "gs_sort_static")
    return keys, vals, ranges, (int(m.value) if count else None)


def sort_status(workspace: torch.Tensor, stream=None):
    """(M, overflowed) of the last gs_sort on this workspace (synchronises)."""
    m = ctypes.c_int64(-1)
    code = L.lib().gs_sort_status(_ptr(workspace), ctypes.byref(m), _stream(stream))
    if code not in (L.GS_OK, L.GS_ERR_CAPACITY):
        L.check(code, "gs_sort_status")
    return int(m.value), code == L.GS_ERR_CAPACITY


def render(splats: torch.Tensor, vals: torch.Tensor, ranges: torch.Tensor, cam, bg=(0.0, 0.0, 0.0),
           out_color=None, final_T=None, n_contrib=None, stream=None):
    """gs_render: returns (image [3, H, W], final_T [H, W], n_contrib [H, W])."""
    dev = splats.device
    H, W = int(cam.height), int(cam.width)
    if out_color is None:
        out_color = torch.empty((3, H, W), dtype=torch.float32, device=dev)
    if final_T is None:
        final_T = torch.empty((H, W), dtype=torch.float32, device=dev)
    if n_contrib is None:
        n_contrib = torch.empty((H, W), dtype=torch.int32, device=dev)
    for t, dt, nm in ((out_color, torch.float32, "out_color"), (final_T, torch.float32, "final_T"),
                      (n_contrib, torch.int32, "n_contrib")):
        _check_tensor(t, dt, nm)
    c = camera_struct(cam)
    bgc = (ctypes.c_float * 3)(*[float(v) for v in bg])
    code = L.lib().gs_render(_ptr(splats), _ptr(vals), _ptr(ranges), ctypes.byref(c), bgc, _ptr(out_color),
                             _ptr(final_T), _ptr(n_contrib), _stream(stream))
    L.check(code, "gs_render")
    return out_color, final_T, n_contrib


def render_contrib(splats: torch.Tensor, vals: torch.Tensor, ranges: torch.Tensor, cam, bg=(0.0, 0.0, 0.0),
                   out_color=None, final_T=None, n_contrib=None, stream=None):
    """gs_render_contrib: the contribution-aware (Seele-style) render; the
    same outputs as render(), bit for bit."""
    dev = splats.device
    H, W = int(cam.height), int(cam.width)
    if out_color is None:
        out_color = torch.empty((3, H, W), dtype=torch.float32, device=dev)
    if final_T is None:
        final_T = torch.empty((H, W), dtype=torch.float32, device=dev)
    if n_contrib is None:
        n_contrib = torch.empty((H, W), dtype=torch.int32, device=dev)
    c = camera_struct(cam)
    bgc = (ctypes.c_float * 3)(*[float(v) for v in bg])
    L.check(L.lib().gs_render_contrib(_ptr(splats), _ptr(vals), _ptr(ranges), ctypes.byref(c), bgc, _ptr(out_color),
                                      _ptr(final_T), _ptr(n_contrib), _stream(stream)), "gs_render_contrib")
    return out_color, final_T, n_contrib


def render_workload(splats: torch.Tensor, vals: torch.Tensor, ranges: torch.Tensor, cam, bg=(0.0, 0.0, 0.0),
                    stream=None, tile_cycles: bool = False):
    """gs_render_workload: (image, final_T, n_contrib, n_eval [H, W] int32),
    plus the per-tile SM cycles [tiles_y, tiles_x] int64 if tile_cycles."""
    dev = splats.device
    H, W = int(cam.height), int(cam.width)
    out_color = torch.empty((3, H, W), dtype=torch.float32, device=dev)
    final_T = torch.empty((H, W), dtype=torch.float32, device=dev)
    n_contrib = torch.empty((H, W), dtype=torch.int32, device=dev)
    n_eval = torch.empty((H, W), dtype=torch.int32, device=dev)
    cyc = None
    if tile_cycles:
        cyc = torch.zeros(((H + 15) // 16, (W + 15) // 16), dtype=torch.int32, device=dev)
    c = camera_struct(cam)
    bgc = (ctypes.c_float * 3)(*[float(v) for v in bg])
    code = L.lib().gs_render_workload(_ptr(splats), _ptr(vals), _ptr(ranges), ctypes.byref(c), bgc,
                                      _ptr(out_color), _ptr(final_T), _ptr(n_contrib), _ptr(n_eval),
                                      _ptr(cyc), _stream(stream))
    L.check(code, "gs_render_workload")
    if tile_cycles:
        # stored as uint32 bit patterns
        return out_color, final_T, n_contrib, n_eval, cyc.to(torch.int64) & 0xFFFFFFFF
    return out_color, final_T, n_contrib, n_eval


def render_invdepth(splats: torch.Tensor, vals: torch.Tensor, ranges: torch.Tensor, cam, bg=(0.0, 0.0, 0.0),
                    stream=None):
    """gs_render_ex with the inverse-depth output: (image, final_T,
    n_contrib, invdepth [H, W] float32)."""
    dev = splats.device
    H, W = int(cam.height), int(cam.width)
    out_color = torch.empty((3, H, W), dtype=torch.float32, device=dev)
    final_T = torch.empty((H, W), dtype=torch.float32, device=dev)
    n_contrib = torch.empty((H, W), dtype=torch.int32, device=dev)
    invdepth = torch.empty((H, W), dtype=torch.float32, device=dev)
    c = camera_struct(cam)
    bgc = (ctypes.c_float * 3)(*[float(v) for v in bg])
    code = L.lib().gs_render_ex(_ptr(splats), _ptr(vals), _ptr(ranges), ctypes.byref(c), bgc, _ptr(out_color),
                                _ptr(final_T), _ptr(n_contrib), _ptr(invdepth), None, None, _stream(stream))
    L.check(code, "gs_render_ex")
    return out_color, final_T, n_contrib, invdepth


class Renderer:
    """Device buffers for rendering one scene size at one resolution.

    ``frame`` enqueues preprocess, sort and render on the current stream
    without any host synchronisation; ``instances`` reads the device-side M
    of the last frame (and whether it overflowed ``m_cap``)."""

    def __init__(self, n: int, width: int, height: int, m_cap: int, device="cuda"):
        self.n, self.width, self.height, self.m_cap = int(n), int(width), int(height), int(m_cap)
        T = ((self.width + 15) // 16) * ((self.height + 15) // 16)
        dev = torch.device(device)
        self.splats = splat_buffer(self.n, dev)
        self.keys = torch.empty(max(self.m_cap, 1), dtype=torch.int64, device=dev)
        self.vals = torch.empty(max(self.m_cap, 1), dtype=torch.int32, device=dev)
        self.ranges = torch.empty((T, 2), dtype=torch.int32, device=dev)
        self.workspace = torch.empty(sort_workspace_bytes(self.n, self.m_cap, T), dtype=torch.uint8, device=dev)
        self.image = torch.empty((3, self.height, self.width), dtype=torch.float32, device=dev)
        self.final_T = torch.empty((self.height, self.width), dtype=torch.float32, device=dev)
        self.n_contrib = torch.empty((self.height, self.width), dtype=torch.int32, device=dev)
        self._ptrs = [_ptr(t) for t in (self.splats, self.keys, self.vals, self.ranges, self.workspace, self.image,
                                        self.final_T, self.n_contrib)]
        self._ws_bytes = self.workspace.numel()
        self._scene_key, self._scene_struct = None, None

    def frame(self, scene: SceneTensors, cam, bg=(0.0, 0.0, 0.0), stream=None):
        """gs_frame: preprocess, sort and render in one call, no host sync."""
        if scene.n != self.n or int(cam.width) != self.width or int(cam.height) != self.height:
            raise ValueError("scene size or resolution differs from the Renderer's buffers")
        key = (id(scene), scene.sh_degree) + tuple(int(t.data_ptr()) for t in
                                                   (scene.means, scene.log_scales, scene.quats,
                                                    scene.opacity_logits, scene.sh))
        if self._scene_key != key:  # validate and build the scene struct once per scene
            self._scene_struct, self._scene_key = scene.struct(), key
        c = camera_struct(cam)
        bgc = (ctypes.c_float * 3)(float(bg[0]), float(bg[1]), float(bg[2]))
        p = self._ptrs
        L.check(L.lib().gs_frame(ctypes.byref(self._scene_struct), ctypes.byref(c), p[0], p[1], p[2], self.m_cap,
                                 p[3], p[4], self._ws_bytes, bgc, p[5], p[6], p[7], _stream(stream)), "gs_frame")
        return self.image, self.final_T, self.n_contrib

    def instances(self, stream=None):
        return sort_status(self.workspace, stream)


JOB_DTYPE = np.dtype([("splats", "<u8"), ("vals", "<u8"), ("ranges", "<u8"), ("out", "<u8"), ("T", "<u8"),
                      ("nc", "<u8"), ("w", "<i4"), ("h", "<i4"), ("bg", "<f4", 3), ("tile_begin", "<u4")])
DESC_HEADER = 16
assert JOB_DTYPE.itemsize == 72  # gs_render_job


@dataclass
class BatchJob:
    """One job of a batched render: gs_render's inputs and outputs."""
    splats: torch.Tensor
    vals: torch.Tensor
    ranges: torch.Tensor
    image: torch.Tensor
    final_T: torch.Tensor
    n_contrib: torch.Tensor
    width: int
    height: int
    bg: tuple = (0.0, 0.0, 0.0)


class RenderBatch:
    """The job table of gs_render_batch / gs_render_batch_split (a
    gs_render_batch_desc) in pinned host memory and on the device, plus the
    work counter.  ``set_jobs`` writes the table and enqueues its upload;
    the launches read it on the device, so a captured launch serves any
    later table."""

    def __init__(self, max_jobs: int, device="cuda"):
        self.max_jobs = int(max_jobs)
        nbytes = DESC_HEADER + JOB_DTYPE.itemsize * self.max_jobs
        self.desc_host = torch.zeros(nbytes, dtype=torch.uint8).pin_memory()
        self.desc_dev = torch.zeros(nbytes, dtype=torch.uint8, device=device)
        self.counter = torch.zeros(1, dtype=torch.int32, device=device)
        self.total_tiles = 0

    def write(self, jobs) -> int:
        """Writes the host table (jobs: BatchJob-like objects); returns the
        total tile count.  Does not upload."""
        if len(jobs) > self.max_jobs:
            raise ValueError(f"{len(jobs)} jobs exceed the table's {self.max_jobs}")
        tab = np.zeros(len(jobs), dtype=JOB_DTYPE)
        total = 0
        for i, j in enumerate(jobs):
            w, h = int(j.width), int(j.height)
            tab[i] = (j.splats.data_ptr(), j.vals.data_ptr(), j.ranges.data_ptr(), j.image.data_ptr(),
                      j.final_T.data_ptr(), j.n_contrib.data_ptr(), w, h, tuple(float(v) for v in j.bg), total)
            total += ((w + 15) // 16) * ((h + 15) // 16)
        host = self.desc_host.numpy()
        host[:8] = np.frombuffer(np.array([len(jobs), total], dtype=np.uint32).tobytes(), np.uint8)
        host[8:DESC_HEADER] = 0
        host[DESC_HEADER:DESC_HEADER + JOB_DTYPE.itemsize * len(jobs)] = np.frombuffer(tab.tobytes(), np.uint8)
        self.total_tiles = total
        return total

    def upload(self, stream=None):
        s = torch.cuda.current_stream() if stream is None else stream
        with torch.cuda.stream(s):
            self.desc_dev.copy_(self.desc_host, non_blocking=True)

    def set_jobs(self, jobs, stream=None) -> int:
        total = self.write(jobs)
        self.upload(stream)
        return total

    def launch(self, grid: int = 0, stream=None):
        """gs_render_batch over the uploaded table."""
        L.check(L.lib().gs_render_batch(_ptr(self.desc_dev), _ptr(self.counter), int(grid), _stream(stream)),
                "gs_render_batch")

    def launch_balanced(self, params: "BalanceParams", workspace: torch.Tensor, grid: int = 0, stream=None):
        """gs_render_batch_balanced over the uploaded table (workspace from
        balance_workspace(params))."""
        _check_tensor(workspace, torch.uint8, "workspace")
        c = params.struct()
        L.check(L.lib().gs_render_batch_balanced(_ptr(self.desc_dev), _ptr(self.counter), ctypes.byref(c),
                                                 _ptr(workspace), workspace.numel(), int(grid), _stream(stream)),
                "gs_render_batch_balanced")


@dataclass
class BalanceParams:
    """gs_balance_params: long-list tiles first (heavy_len splats and up,
    0 = off) and splitting of tiles still live after `budget` splats
    (0 = off) into max_chunks chunks of `chunk` splats."""
    heavy_len: int = 4096
    max_heavy_tiles: int = 4096
    budget: int = 0
    max_split_tiles: int = 0
    max_chunks: int = 32
    chunk: int = 1024

    def struct(self) -> L.GsBalanceParams:
        return L.GsBalanceParams(int(self.heavy_len), int(self.max_heavy_tiles), int(self.budget),
                                 int(self.max_split_tiles), int(self.max_chunks), int(self.chunk))


def balance_workspace(params: BalanceParams, device="cuda") -> torch.Tensor:
    c = params.struct()
    n = int(L.lib().gs_render_balance_workspace_bytes(ctypes.byref(c)))
    if n == 0:
        raise ValueError(f"invalid balance parameters {params}")
    return torch.empty(n, dtype=torch.uint8, device=device)


class FramePipeline:
    """End-to-end frames from host memory, double-buffered.

    Each ``submit`` uploads a scene from pinned host memory, renders it and
    reads the image back to pinned host memory -- every step of a frame,
    every frame -- but on three streams: the upload of frame k+1 runs while
    frame k renders, and the read-back of frame k runs while frame k+1 is
    uploaded.  Two slots (device scene, Renderer, host image) alternate; a
    slot is reused only after its previous frame's image has been read back.
    The host-to-device link, not the GPU, bounds the rate for large scenes.
    """

    class _Slot:
        def __init__(self, n, width, height, m_cap, device):
            f = lambda *shape: torch.empty(shape, dtype=torch.float32, device=device)
            self.scene = SceneTensors(f(n, 3), f(n, 3), f(n, 4), f(n), f(n, 16, 3))
            self.renderer = Renderer(n, width, height, m_cap, device)
            self.host_image = torch.empty((3, height, width), dtype=torch.float32).pin_memory()
            self.h2d_done = torch.cuda.Event()
            self.d2h_done = torch.cuda.Event()
            self.ticket = -1

    def __init__(self, n: int, width: int, height: int, m_cap: int, device="cuda"):
        self.device = torch.device(device)
        self.slots = [self._Slot(int(n), int(width), int(height), int(m_cap), self.device) for _ in range(2)]
        self.h2d = torch.cuda.Stream(self.device)
        self.compute = torch.cuda.Stream(self.device)
        self.d2h = torch.cuda.Stream(self.device)
        self.k = 0

    def submit(self, host_arrays, cam, bg=(0.0, 0.0, 0.0), sh_degree: int = 3) -> int:
        """Enqueue one frame.  host_arrays: pinned CPU tensors (means,
        log_scales, quats, opacity_logits, sh), kept unchanged until the
        frame's upload has run.  Returns a ticket for ``result``."""
        slot = self.slots[self.k % 2]
        dst = [slot.scene.means, slot.scene.log_scales, slot.scene.quats, slot.scene.opacity_logits, slot.scene.sh]
        slot.scene.sh_degree = int(sh_degree)
        self.h2d.wait_event(slot.d2h_done)  # the slot's previous frame is finished and read back
        with torch.cuda.stream(self.h2d):
            for d, h in zip(dst, host_arrays):
                if not h.is_pinned() or h.shape != d.shape or h.dtype != torch.float32:
                    raise ValueError("host arrays must be pinned float32 tensors of the pipeline's scene size")
                d.copy_(h, non_blocking=True)
            slot.h2d_done.record(self.h2d)
        self.compute.wait_event(slot.h2d_done)
        with torch.cuda.stream(self.compute):
            image, _, _ = slot.renderer.frame(slot.scene, cam, bg)
            done = torch.cuda.Event()
            done.record(self.compute)
        self.d2h.wait_event(done)
        with torch.cuda.stream(self.d2h):
            slot.host_image.copy_(image, non_blocking=True)
            slot.d2h_done.record(self.d2h)
        slot.ticket = self.k
        self.k += 1
        return slot.ticket

    def result(self, ticket: int) -> torch.Tensor:
        """The host image of frame ``ticket`` (waits for it).  Valid until
        the frame two submits later reuses the slot."""
        slot = self.slots[ticket % 2]
        if slot.ticket != ticket:
            raise ValueError("frame already overwritten (only the last two frames are kept)")
        slot.d2h_done.synchronize()
        return slot.host_image

    def instances(self, ticket: int):
        """(M, overflow) of frame ``ticket`` (synchronises)."""
        slot = self.slots[ticket % 2]
        slot.d2h_done.synchronize()
        return slot.renderer.instances()


def render_backward(scene: SceneTensors, cam, splats, vals, ranges, final_T, n_contrib, dL_dcolor,
                    bg=(0.0, 0.0, 0.0), workspace=None, stream=None):
    """gs_render_backward: gradients of sum(dL_dcolor * image) with respect to
    the scene tensors, as a dict; also the per-splat 2D gradients [n, 12]."""
    dev = splats.device
    n = scene.n
    grads = {k: torch.empty_like(getattr(scene, k)) for k in ("means", "log_scales", "quats", "opacity_logits",
                                                                  "sh")}
    need = int(L.lib().gs_backward_workspace_bytes(n))
    if workspace is None:
        workspace = torch.empty(need // 4, dtype=torch.float32, device=dev)
    dL = dL_dcolor.contiguous().to(torch.float32)
    _check_tensor(dL, torch.float32, "dL_dcolor")
    g = L.GsSceneGrads()
    g.dmeans, g.dlog_scales, g.dquats = grads["means"].data_ptr(), grads["log_scales"].data_ptr(), \
        grads["quats"].data_ptr()
    g.dopacity_logits, g.dsh = grads["opacity_logits"].data_ptr(), grads["sh"].data_ptr()
    c = camera_struct(cam)
    bgc = (ctypes.c_float * 3)(*[float(v) for v in bg])
    code = L.lib().gs_render_backward(ctypes.byref(scene.struct()), ctypes.byref(c), _ptr(splats), _ptr(vals),
                                      _ptr(ranges), bgc, _ptr(final_T), _ptr(n_contrib), _ptr(dL), _ptr(workspace),
                                      workspace.numel() * 4, ctypes.byref(g), _stream(stream))
    L.check(code, "gs_render_backward")
    return grads, workspace.view(-1, 12)[:max(n, 1)]


def render_backward_splats(cam, splats, n, vals, ranges, final_T, n_contrib, dL_dcolor, bg=(0.0, 0.0, 0.0),
                           dsplat=None, stream=None):
    """gs_render_backward_splats: the per-splat 2D gradients [n, 12]
    (dL/d x, y, conic a, b, c, opacity, r, g, b; 3 unused)."""
    n = int(n)
    if dsplat is None:
        dsplat = torch.empty((max(n, 1), 12), dtype=torch.float32, device=splats.device)
    _check_tensor(dsplat, torch.float32, "dsplat")
    dL = dL_dcolor.contiguous().to(torch.float32)
    _check_tensor(dL, torch.float32, "dL_dcolor")
    c = camera_struct(cam)
    bgc = (ctypes.c_float * 3)(*[float(v) for v in bg])
    L.check(L.lib().gs_render_backward_splats(ctypes.byref(c), _ptr(splats), n, _ptr(vals), _ptr(ranges), bgc,
                                              _ptr(final_T), _ptr(n_contrib), _ptr(dL), _ptr(dsplat),
                                              _stream(stream)), "gs_render_backward_splats")
    return dsplat


def preprocess_backward(scene: SceneTensors, cam, splats, dsplat, grads=None, stream=None):
    """gs_preprocess_backward: the scene gradients (a dict like
    render_backward's) from the per-splat 2D gradients."""
    if grads is None:
        grads = {k: torch.empty_like(getattr(scene, k)) for k in ("means", "log_scales", "quats", "opacity_logits",
                                                                      "sh")}
    _check_tensor(dsplat, torch.float32, "dsplat")
    g = L.GsSceneGrads()
    g.dmeans, g.dlog_scales, g.dquats = grads["means"].data_ptr(), grads["log_scales"].data_ptr(), \
        grads["quats"].data_ptr()
    g.dopacity_logits, g.dsh = grads["opacity_logits"].data_ptr(), grads["sh"].data_ptr()
    c = camera_struct(cam)
    L.check(L.lib().gs_preprocess_backward(ctypes.byref(scene.struct()), ctypes.byref(c), _ptr(splats),
                                           _ptr(dsplat), ctypes.byref(g), _stream(stream)), "gs_preprocess_backward")
    return grads


class RasterizeGaussians(torch.autograd.Function):
    """image = render(preprocess(scene), sort) with the CUDA backward.

    forward(means, log_scales, quats, opacity_logits, sh, cam, bg, sh_degree)
    -> image [3, H, W].  The sort's instance count is read once per call (one
    host synchronisation) to size the key buffers."""

    @staticmethod
    def forward(ctx, means, log_scales, quats, opacity_logits, sh, cam, bg=(0.0, 0.0, 0.0), sh_degree=3):
        scene = SceneTensors(means.detach().contiguous(), log_scales.detach().contiguous(),
                             quats.detach().contiguous(), opacity_logits.detach().contiguous(),
                             sh.detach().contiguous(), int(sh_degree))
        splats = preprocess(scene, cam)
        cap = max(1024, 8 * scene.n)
        try:
            keys, vals, ranges, m, _ = sort(splats, scene.n, cam, cap)
        except L.GsError as e:
            if e.code != L.GS_ERR_CAPACITY:
                raise
            keys, vals, ranges, m, _ = sort(splats, scene.n, cam, e.m)
        img, final_T, n_contrib = render(splats, vals, ranges, cam, bg)
        ctx.save_for_backward(scene.means, scene.log_scales, scene.quats, scene.opacity_logits, scene.sh, splats,
                              vals, ranges, final_T, n_contrib)
        ctx.cam, ctx.bg, ctx.sh_degree = cam, tuple(bg), int(sh_degree)
        return img

    @staticmethod
    def backward(ctx, dL_dimg):
        means, log_scales, quats, logits, sh, splats, vals, ranges, final_T, n_contrib = ctx.saved_tensors
        scene = SceneTensors(means, log_scales, quats, logits, sh, ctx.sh_degree)
        grads, _ = render_backward(scene, ctx.cam, splats, vals, ranges, final_T, n_contrib, dL_dimg, ctx.bg)
        return (grads["means"], grads["log_scales"], grads["quats"], grads["opacity_logits"], grads["sh"], None,
                None, None)


def rasterize(means, log_scales, quats, opacity_logits, sh, cam, bg=(0.0, 0.0, 0.0), sh_degree=3):
    """Differentiable render of a scene (see RasterizeGaussians)."""
    return RasterizeGaussians.apply(means, log_scales, quats, opacity_logits, sh, cam, bg, sh_degree)
