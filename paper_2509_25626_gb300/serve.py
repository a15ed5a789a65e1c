"""Continuous-batching render server over resident scenes.

Requests (scene, camera) arrive over time.  Each is admitted when a slot
and enough device memory (by a per-(scene, resolution) estimate) are free;
its preprocess and sort then run at once on a stream of their own, so they
overlap whatever batch is rendering.  Whenever the render engine is idle,
every admitted request joins one batch, rendered by a single persistent
launch (gs_render_batch) replayed from a captured CUDA graph; the launch
waits for those requests' sorts on the device, not on the host.  A request
is complete when its batch's render has finished; its latency is completion
time minus arrival time.

Every kernel runs in libgs.so; this module only schedules, allocates (from
PyTorch's caching allocator) and keeps time.
"""

from __future__ import annotations

import collections
import ctypes
import dataclasses
import math
import time

import numpy as np
import torch

from . import _lib as L
from .api import SceneTensors, camera_struct, num_tiles, preprocess, render, sort, sort_workspace_bytes, splat_buffer

JOB_BYTES = 72
DESC_HEADER = 16


@dataclasses.dataclass
class Request:
    rid: int
    arrival: float          # seconds from the start of the run
    scene: str
    cam: object
    bg: tuple = (0.0, 0.0, 0.0)
    # filled in by the server
    t_admit: float = math.nan
    t_done: float = math.nan
    image: torch.Tensor | None = None
    final_T: torch.Tensor | None = None
    n_contrib: torch.Tensor | None = None
    instances: int = -1

    @property
    def latency(self) -> float:
        return self.t_done - self.arrival


class _Slot:
    """Device buffers of one in-flight request."""

    def __init__(self, n, cam, m_cap, device):
        T = num_tiles(cam)
        H, W = int(cam.height), int(cam.width)
        self.splats = splat_buffer(n, device)
        self.keys = torch.empty(max(m_cap, 1), dtype=torch.int64, device=device)
        self.vals = torch.empty(max(m_cap, 1), dtype=torch.int32, device=device)
        self.ranges = torch.empty((T, 2), dtype=torch.int32, device=device)
        self.workspace = torch.empty(sort_workspace_bytes(n, m_cap, T), dtype=torch.uint8, device=device)
        self.image = torch.empty((3, H, W), dtype=torch.float32, device=device)
        self.final_T = torch.empty((H, W), dtype=torch.float32, device=device)
        self.n_contrib = torch.empty((H, W), dtype=torch.int32, device=device)
        self.header = torch.empty(4, dtype=torch.int64).pin_memory()   # m_total, nvis|m_sort, overflow|timeout
        self.m_cap = m_cap
        self.tiles = T

    @staticmethod
    def bytes_for(n, cam, m_cap) -> int:
        T = num_tiles(cam)
        px = int(cam.width) * int(cam.height)
        return 64 * max(n, 1) + 12 * max(m_cap, 1) + 8 * T + sort_workspace_bytes(n, m_cap, T) + 20 * px


class Server:
    """scenes: name -> SceneTensors (resident).  m_caps: (scene, width,
    height) -> instance capacity per request (see ``calibrate``)."""

    def __init__(self, scenes: dict, max_batch: int = 16, mem_budget: int = 24 << 30, device="cuda",
                 n_streams: int = 8, use_graph: bool = True):
        self.scenes = scenes
        self.device = torch.device(device)
        self.max_batch = max_batch
        self.mem_budget = mem_budget
        self.m_caps = {}
        self.streams = [torch.cuda.Stream(self.device) for _ in range(n_streams)]
        self.render_stream = torch.cuda.Stream(self.device)
        cap_desc = DESC_HEADER + JOB_BYTES * max_batch
        self.desc_host = torch.zeros(cap_desc, dtype=torch.uint8).pin_memory()
        self.desc_dev = torch.zeros(cap_desc, dtype=torch.uint8, device=self.device)
        self.counter = torch.zeros(1, dtype=torch.int32, device=self.device)
        self.use_graph = use_graph
        self.graph = None
        self.stats = collections.Counter()

    # ------------------------------------------------------------------ setup
    def calibrate(self, scene: str, width: int, height: int, cams, margin: float = 1.5):
        """Instance capacity for a (scene, resolution) from the sorts of a
        few sample poses."""
        st = self.scenes[scene]
        m = 0
        for cam in cams:
            sp = preprocess(st, cam)
            cap = 1 << 22
            while True:
                try:
                    _, _, _, mm, _ = sort(sp, st.n, cam, cap)
                    break
                except L.GsError as e:
                    if e.code != L.GS_ERR_CAPACITY:
                        raise
                    cap = max(2 * cap, getattr(e, "m", 0) + 1)
            m = max(m, mm)
        self.m_caps[(scene, width, height)] = int(m * margin) + 4096
        torch.cuda.synchronize(self.device)

    def _graph_launch(self):
        lib = L.lib()
        s = ctypes.c_void_p(int(torch.cuda.current_stream(self.device).cuda_stream))
        L.check(lib.gs_render_batch(ctypes.c_void_p(self.desc_dev.data_ptr()),
                                    ctypes.c_void_p(self.counter.data_ptr()), 0, s), "gs_render_batch")

    def _ensure_graph(self):
        if self.graph is not None or not self.use_graph:
            return
        # an empty batch, then capture the launch (memset + persistent kernel)
        self.desc_host.zero_()
        self.desc_dev.copy_(self.desc_host)
        torch.cuda.synchronize(self.device)
        with torch.cuda.stream(self.render_stream):
            self._graph_launch()  # warm-up outside the capture
        torch.cuda.synchronize(self.device)
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=self.render_stream):
            self._graph_launch()
        self.graph = g
        torch.cuda.synchronize(self.device)

    # -------------------------------------------------------------- requests
    def _admit(self, req: Request, stream: torch.cuda.Stream):
        st = self.scenes[req.scene]
        key = (req.scene, int(req.cam.width), int(req.cam.height))
        m_cap = self.m_caps[key]
        with torch.cuda.stream(stream):
            slot = _Slot(st.n, req.cam, m_cap, self.device)
            preprocess(st, req.cam, slot.splats, stream=stream)
            sort(slot.splats, st.n, req.cam, m_cap, slot.keys, slot.vals, slot.ranges, slot.workspace, count=False,
                 stream=stream)
            slot.header.copy_(slot.workspace[:32].view(torch.int64), non_blocking=True)
            ev = torch.cuda.Event()
            ev.record(stream)
        return slot, ev

    def _write_desc(self, batch):
        host = self.desc_host.numpy()
        total = 0
        jobs = np.zeros(len(batch), dtype=np.dtype([("splats", "<u8"), ("vals", "<u8"), ("ranges", "<u8"),
                                                    ("out", "<u8"), ("T", "<u8"), ("nc", "<u8"), ("w", "<i4"),
                                                    ("h", "<i4"), ("bg", "<f4", 3), ("tile_begin", "<u4")]))
        for i, (req, slot) in enumerate(batch):
            jobs[i] = (slot.splats.data_ptr(), slot.vals.data_ptr(), slot.ranges.data_ptr(), slot.image.data_ptr(),
                       slot.final_T.data_ptr(), slot.n_contrib.data_ptr(), int(req.cam.width), int(req.cam.height),
                       req.bg, total)
            total += slot.tiles
        assert jobs.dtype.itemsize == JOB_BYTES
        hdr = np.zeros(DESC_HEADER, np.uint8)
        hdr[:8] = np.frombuffer(np.array([len(batch), total], dtype=np.uint32).tobytes(), np.uint8)
        host[:DESC_HEADER] = hdr
        host[DESC_HEADER:DESC_HEADER + JOB_BYTES * len(batch)] = np.frombuffer(jobs.tobytes(), np.uint8)
        return total

    def serve(self, requests: list[Request], realtime: bool = True):
        """Serves the requests (sorted by arrival).  With realtime=False all
        requests are present at t = 0 (a saturation run)."""
        self._ensure_graph()
        pending = collections.deque(sorted(requests, key=lambda r: r.arrival))
        prepared = []             # (req, slot, event)
        rendering = None          # (batch, event)
        mem_used = 0
        sidx = 0
        t0 = time.perf_counter()
        now = lambda: time.perf_counter() - t0
        done = []
        while pending or prepared or rendering:
            t = now()
            # admission: arrived requests while a slot and memory are free
            while pending and (not realtime or pending[0].arrival <= t) and \
                    len(prepared) + (len(rendering[0]) if rendering else 0) < 2 * self.max_batch:
                req = pending[0]
                key = (req.scene, int(req.cam.width), int(req.cam.height))
                need = _Slot.bytes_for(self.scenes[req.scene].n, req.cam, self.m_caps[key])
                if mem_used + need > self.mem_budget and (prepared or rendering):
                    self.stats["admission_waits"] += 1
                    break
                pending.popleft()
                req.t_admit = now()
                slot, ev = self._admit(req, self.streams[sidx % len(self.streams)])
                sidx += 1
                mem_used += need
                prepared.append((req, slot, ev, need))
            # completion of the batch in flight
            if rendering and rendering[1].query():
                tdone = now()
                for req, slot, _, need in rendering[0]:
                    req.t_done = tdone
                    req.image, req.final_T, req.n_contrib = slot.image, slot.final_T, slot.n_contrib
                    req.instances = int(slot.header[0])
                    if int(slot.header[2]) != 0:  # overflow | timeout << 32
                        self.stats["overflow_or_timeout"] += 1
                    mem_used -= need
                    done.append(req)
                self.stats["batches"] += 1
                rendering = None
            # launch a batch of the prepared requests as soon as the render
            # engine is free: the render stream waits for their sorts on the
            # device, so no host round trip sits between a sort and its render
            if rendering is None and prepared:
                ready = prepared
                if ready:
                    batch = ready[: self.max_batch]
                    for b in batch:
                        prepared.remove(b)
                    total = self._write_desc([(r, s) for r, s, _, _ in batch])
                    rs = self.render_stream
                    for _, _, ev, _ in batch:
                        rs.wait_event(ev)
                    with torch.cuda.stream(rs):
                        self.desc_dev.copy_(self.desc_host, non_blocking=True)
                        if self.graph is not None:
                            self.graph.replay()
                        else:
                            self._graph_launch()
                        ev = torch.cuda.Event()
                        ev.record(rs)
                    self.stats["jobs"] += len(batch)
                    self.stats["tiles"] += total
                    rendering = (batch, ev)
            if not (rendering or prepared) and pending and realtime:
                wait = pending[0].arrival - now()
                if wait > 0:
                    time.sleep(min(wait, 1e-3))
        wall = now()
        torch.cuda.synchronize(self.device)
        return done, wall

    def serve_sequential(self, requests: list[Request], realtime: bool = True):
        """One request at a time: preprocess, sort, render, wait; FIFO."""
        order = sorted(requests, key=lambda r: r.arrival)
        t0 = time.perf_counter()
        now = lambda: time.perf_counter() - t0
        stream = self.streams[0]
        for req in order:
            if realtime:
                wait = req.arrival - now()
                if wait > 0:
                    time.sleep(wait)
            req.t_admit = now()
            st = self.scenes[req.scene]
            key = (req.scene, int(req.cam.width), int(req.cam.height))
            with torch.cuda.stream(stream):
                slot = _Slot(st.n, req.cam, self.m_caps[key], self.device)
                preprocess(st, req.cam, slot.splats, stream=stream)
                sort(slot.splats, st.n, req.cam, slot.m_cap, slot.keys, slot.vals, slot.ranges, slot.workspace,
                     count=False, stream=stream)
                render(slot.splats, slot.vals, slot.ranges, req.cam, req.bg, slot.image, slot.final_T,
                       slot.n_contrib, stream=stream)
            stream.synchronize()
            req.t_done = now()
            req.image, req.final_T, req.n_contrib = slot.image, slot.final_T, slot.n_contrib
        return order, now()


def poisson_requests(rate: float, duration: float, scenes: list[str], resolutions: list[tuple], cam_fn, seed: int = 0):
    """Request stream with exponential inter-arrival times (rate per second),
    uniform scene and resolution, and a random orbit pose from cam_fn(k, w, h)."""
    rng = np.random.default_rng(seed)
    t, out = 0.0, []
    while True:
        t += rng.exponential(1.0 / rate)
        if t > duration:
            break
        w, h = resolutions[rng.integers(len(resolutions))]
        out.append(Request(len(out), t, scenes[rng.integers(len(scenes))], cam_fn(rng.uniform(0, 1), w, h)))
    return out


def latency_stats(done: list[Request], wall: float) -> dict:
    lat = np.array([r.latency for r in done]) * 1000.0
    return dict(requests=len(done), p50_ms=float(np.percentile(lat, 50)), p99_ms=float(np.percentile(lat, 99)),
                mean_ms=float(lat.mean()), frames_per_s=len(done) / wall, wall_s=wall)
