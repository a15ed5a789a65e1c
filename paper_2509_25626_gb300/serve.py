"""Continuous-batching render server over resident scenes.

Requests (scene, camera) arrive over time.  Device memory is divided up
front into request slots, per scene: each slot holds the splat buffer, the
sort's keys, values, ranges and workspace for that scene at the largest
calibrated resolution, a device camera block, and a CUDA stream.  A request
is admitted as soon as a slot of its scene is free (memory-based admission:
the slots are the memory).  Its preprocess and sort run at once on the
slot's stream by replaying a CUDA graph captured for that slot and
resolution -- the camera goes in through the slot's camera block, which the
graph copies from pinned host memory before the preprocess -- so they
overlap whatever batch is rendering.  Whenever the render engine is idle,
every prepared request joins one batch, rendered by a single persistent
launch (gs_render_batch) replayed from a captured graph; the launch waits
for those requests' sorts on the device, not on the host.  A request is
complete when its batch's render has finished; its latency is completion
time minus arrival time.  A request whose tile instances overflowed its
slot's capacity (or whose sort reported a timeout) is returned as failed,
with no image, and is left out of the latency statistics.

Every kernel runs in libgs.so; this module only schedules, owns the
preallocated buffers, and keeps time.  Each request's outputs (image,
final T, n_contrib) are tensors of its own, handed to the caller.
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
from .api import (BatchJob, RenderBatch, SceneTensors, _ptr, camera_struct, num_tiles, preprocess, render, sort,
                  sort_workspace_bytes, splat_buffer)

# 16-byte aligned room for the kernels' camera block
CAM_BLOCK_BYTES = 128


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
    error: str | None = None  # "capacity" or "timeout" for a failed request

    @property
    def latency(self) -> float:
        return self.t_done - self.arrival


class _Slot:
    """The preallocated buffers of one in-flight request of a scene."""

    def __init__(self, scene: str, n: int, m_cap: int, max_tiles: int, device):
        self.scene, self.n, self.m_cap = scene, int(n), int(m_cap)
        self.splats = splat_buffer(n, device)
        self.keys = torch.empty(max(m_cap, 1), dtype=torch.int64, device=device)
        self.vals = torch.empty(max(m_cap, 1), dtype=torch.int32, device=device)
        self.ranges = torch.empty((max_tiles, 2), dtype=torch.int32, device=device)
        self.workspace = torch.empty(sort_workspace_bytes(n, m_cap, max_tiles), dtype=torch.uint8, device=device)
        self.cam_dev = torch.zeros(CAM_BLOCK_BYTES, dtype=torch.uint8, device=device)
        self.cam_host = torch.zeros(CAM_BLOCK_BYTES, dtype=torch.uint8).pin_memory()
        self.header = torch.zeros(4, dtype=torch.int64).pin_memory()  # m_total, nvis|m_sort, overflow|timeout
        self.stream = torch.cuda.Stream(device)
        self.graphs = {}  # (width, height) -> captured preprocess + sort
        self.done_event = None

    @staticmethod
    def bytes_for(n: int, m_cap: int, max_tiles: int) -> int:
        return 80 * max(n, 1) + 12 * max(m_cap, 1) + 8 * max_tiles + sort_workspace_bytes(n, m_cap, max_tiles)

    def set_camera(self, cam):
        c = camera_struct(cam)
        L.check(L.lib().gs_camera_block(ctypes.byref(c), ctypes.c_void_p(self.cam_host.data_ptr())),
                "gs_camera_block")

    def front(self, st: SceneTensors, cam, stream):
        """Preprocess (camera from the slot's camera block) and sort, no host
        synchronisation; the header of the sort's counters is copied back to
        pinned memory after it."""
        with torch.cuda.stream(stream):
            self.cam_dev.copy_(self.cam_host, non_blocking=True)
            sc = st.struct()
            L.check(L.lib().gs_preprocess_camblock(ctypes.byref(sc), _ptr(self.cam_dev), _ptr(self.splats),
                                                   ctypes.c_void_p(int(stream.cuda_stream))),
                    "gs_preprocess_camblock")
            T = num_tiles(cam)
            sort(self.splats, self.n, cam, self.m_cap, self.keys, self.vals, self.ranges[:T], self.workspace,
                 count=False, stream=stream)
            self.header.copy_(self.workspace[:32].view(torch.int64), non_blocking=True)


class Server:
    """scenes: name -> SceneTensors (resident).  resolutions: the (width,
    height) requests may ask for.  ``calibrate`` every (scene, resolution)
    first; the first ``serve`` call then divides ``mem_budget`` into request
    slots per scene (at most ``slots_per_scene``, at least one) and captures
    each slot's preprocess + sort graph per resolution."""

    def __init__(self, scenes: dict, resolutions=None, max_batch: int = 16, mem_budget: int = 24 << 30,
                 device="cuda", slots_per_scene: int = 8, use_graph: bool = True, render_priority: bool = False,
                 single_direct: bool = True, overlap_min: int = 2, ready_only: bool = True):
        self.scenes = scenes
        self.resolutions = [tuple(r) for r in (resolutions or [])]
        self.device = torch.device(device)
        self.max_batch = max_batch
        self.mem_budget = mem_budget
        self.slots_per_scene = slots_per_scene
        self.use_graph = use_graph
        self.single_direct = single_direct
        # overlap_min: while a request is in flight, arrived requests start
        # their preprocess + sort only once at least this many are waiting.
        # A lone arrival then waits for the GPU as in one-at-a-time serving
        # (its front would otherwise share the SMs with the render in flight
        # and delay both); a queue starts the overlapped, batched pipeline.
        self.overlap_min = max(1, int(overlap_min))
        # ready_only: while few requests are prepared (a short queue), a
        # batch takes those whose preprocess + sort has completed (at least
        # the oldest one), so that a request whose sort is done does not wait
        # for a later arrival's sort; a long queue is batched whole
        self.ready_only = ready_only
        self.ready_only_max = 3
        self.m_caps = {}
        # render_priority: the batch render at the highest stream priority
        # (measured no better for latency at 200 and 800 requests/s)
        prio = torch.cuda.Stream.priority_range()[1] if render_priority else 0
        self.render_stream = torch.cuda.Stream(self.device, priority=prio)
        self.batch = RenderBatch(max_batch, device=self.device)
        self.graph = None
        self.pools = None
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
        if (width, height) not in self.resolutions:
            self.resolutions.append((width, height))
        torch.cuda.synchronize(self.device)

    def _cam_of(self, w, h):
        """A placeholder camera of that size for graph capture (the pose
        comes from the camera block at replay)."""
        class _C:
            pass
        c = _C()
        c.viewmat = np.eye(4, dtype=np.float32)
        c.viewmat[2, 3] = 4.0
        c.fx = c.fy = float(w)
        c.cx, c.cy = (w - 1) / 2.0, (h - 1) / 2.0
        c.width, c.height = int(w), int(h)
        c.tan_fovx, c.tan_fovy = 0.5, 0.5 * h / w
        return c

    def _ensure_ready(self):
        if self.pools is not None:
            return
        max_tiles = max(num_tiles(self._cam_of(w, h)) for w, h in self.resolutions)
        per_scene = self.mem_budget // max(1, len(self.scenes))
        self.pools = {}
        for name, st in self.scenes.items():
            m_cap = max(v for (s, _, _), v in self.m_caps.items() if s == name)
            nbytes = _Slot.bytes_for(st.n, m_cap, max_tiles)
            count = max(1, min(self.slots_per_scene, per_scene // nbytes))
            self.pools[name] = [_Slot(name, st.n, m_cap, max_tiles, self.device) for _ in range(count)]
            self.stats[f"slots_{name}"] = count
        torch.cuda.synchronize(self.device)
        # warm-up outside capture (first calls look up device attributes)
        for name, pool in self.pools.items():
            for w, h in self.resolutions:
                cam = self._cam_of(w, h)
                pool[0].set_camera(cam)
                pool[0].front(self.scenes[name], cam, pool[0].stream)
        self.batch.set_jobs([], stream=self.render_stream)
        with torch.cuda.stream(self.render_stream):
            self.batch.launch(stream=self.render_stream)
        torch.cuda.synchronize(self.device)
        if self.use_graph:
            for name, pool in self.pools.items():
                st = self.scenes[name]
                for slot in pool:
                    for w, h in self.resolutions:
                        g = torch.cuda.CUDAGraph()
                        cam = self._cam_of(w, h)
                        with torch.cuda.graph(g, stream=slot.stream):
                            slot.front(st, cam, slot.stream)
                        slot.graphs[(w, h)] = g
            g = torch.cuda.CUDAGraph()
            with torch.cuda.graph(g, stream=self.render_stream):
                self.batch.upload(stream=self.render_stream)
                self.batch.launch(stream=self.render_stream)
            self.graph = g
        torch.cuda.synchronize(self.device)

    # -------------------------------------------------------------- requests
    def _front(self, req: Request, slot: _Slot):
        slot.set_camera(req.cam)
        key = (int(req.cam.width), int(req.cam.height))
        if self.use_graph:
            with torch.cuda.stream(slot.stream):
                slot.graphs[key].replay()
        else:
            slot.front(self.scenes[req.scene], req.cam, slot.stream)
        ev = torch.cuda.Event()
        ev.record(slot.stream)
        return ev

    def _outputs(self, req: Request):
        H, W = int(req.cam.height), int(req.cam.width)
        dev = self.device
        return (torch.empty((3, H, W), dtype=torch.float32, device=dev),
                torch.empty((H, W), dtype=torch.float32, device=dev),
                torch.empty((H, W), dtype=torch.int32, device=dev))

    def _finish(self, req: Request, slot: _Slot, t_done: float, done: list):
        req.t_done = t_done
        req.instances = int(slot.header[0])
        flags = int(slot.header[2])  # overflow | timeout << 32
        if flags & 0xFFFFFFFF:
            req.error = "capacity"
        elif flags >> 32:
            req.error = "timeout"
        if req.error:
            req.image = req.final_T = req.n_contrib = None
            self.stats["failed"] += 1
        done.append(req)

    def serve(self, requests: list[Request], realtime: bool = True):
        """Serves the requests (sorted by arrival).  With realtime=False all
        requests are present at t = 0 (a saturation run)."""
        self._ensure_ready()
        pending = collections.deque(sorted(requests, key=lambda r: r.arrival))
        free = {name: list(pool) for name, pool in self.pools.items()}
        prepared = []             # (req, slot, event)
        rendering = None          # (batch, event)
        t0 = time.perf_counter()
        now = lambda: time.perf_counter() - t0
        done = []
        while pending or prepared or rendering:
            t = now()
            # admission: arrived requests while a slot of their scene is free;
            # with work in flight, only once overlap_min of them are waiting
            admit = may_admit(pending, t, bool(rendering or prepared), realtime, self.overlap_min)
            while admit and pending and (not realtime or pending[0].arrival <= t):
                req = pending[0]
                if not free[req.scene]:
                    self.stats["admission_waits"] += 1
                    break
                pending.popleft()
                slot = free[req.scene].pop()
                req.t_admit = now()
                prepared.append((req, slot, self._front(req, slot)))
            # completion of the batch in flight
            if rendering and rendering[1].query():
                tdone = now()
                for req, slot, _ in rendering[0]:
                    self._finish(req, slot, tdone, done)
                    free[slot.scene].append(slot)
                self.stats["batches"] += 1
                rendering = None
            # launch a batch of the prepared requests as soon as the render
            # engine is free: the render stream waits for their sorts on the
            # device, so no host round trip sits between a sort and its render
            if rendering is None and prepared:
                take = batch_size([ev for _, _, ev in prepared], self.max_batch,
                                  self.ready_only_max if self.ready_only else 0)
                batch, prepared = prepared[:take], prepared[take:]
                jobs = []
                for req, slot, _ in batch:
                    req.image, req.final_T, req.n_contrib = self._outputs(req)
                    jobs.append(BatchJob(slot.splats, slot.vals, slot.ranges, req.image, req.final_T, req.n_contrib,
                                         req.cam.width, req.cam.height, req.bg))
                rs = self.render_stream
                if len(batch) == 1 and self.single_direct:
                    # a batch of one: gs_render itself (the same blend, bit
                    # for bit), on the request's own stream right after its
                    # sort -- no job table, no cross-stream wait
                    req, slot, _ = batch[0]
                    rs = slot.stream
                else:
                    for _, _, ev in batch:
                        rs.wait_event(ev)
                with torch.cuda.stream(rs):
                    if len(batch) == 1 and self.single_direct:
                        render(slot.splats, slot.vals, slot.ranges[:num_tiles(req.cam)], req.cam, req.bg, req.image,
                               req.final_T, req.n_contrib, stream=rs)
                        total = num_tiles(req.cam)
                    else:
                        total = self.batch.write(jobs)
                        if self.graph is not None:
                            self.graph.replay()
                        else:
                            self.batch.upload(stream=rs)
                            self.batch.launch(stream=rs)
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
        """One request at a time, FIFO, on the same slots and captured
        preprocess + sort: front, gs_render, wait."""
        self._ensure_ready()
        order = sorted(requests, key=lambda r: r.arrival)
        t0 = time.perf_counter()
        now = lambda: time.perf_counter() - t0
        done = []
        for req in order:
            if realtime:
                wait = req.arrival - now()
                if wait > 0:
                    time.sleep(wait)
            req.t_admit = now()
            slot = self.pools[req.scene][0]
            self._front(req, slot)
            req.image, req.final_T, req.n_contrib = self._outputs(req)
            render(slot.splats, slot.vals, slot.ranges[:num_tiles(req.cam)], req.cam, req.bg, req.image,
                   req.final_T, req.n_contrib, stream=slot.stream)
            slot.stream.synchronize()
            self._finish(req, slot, now(), done)
        return done, now()


def may_admit(pending, t: float, in_flight: bool, realtime: bool, overlap_min: int) -> bool:
    """The admission rule of Server.serve: with nothing in flight (or in a
    saturation run) arrived requests are admitted at once; with a request in
    flight, only once at least overlap_min of them have arrived.  pending:
    the requests not yet admitted, by arrival time."""
    if not in_flight or not realtime or overlap_min <= 1:
        return True
    arrived = 0
    for r in pending:
        if r.arrival > t or arrived >= overlap_min:
            break
        arrived += 1
    return arrived >= overlap_min


def batch_size(events, max_batch: int, ready_only_max: int) -> int:
    """How many prepared requests (in admission order; events: their sorts'
    completion events, each with .query()) the next batch takes: up to
    max_batch, and, while at most ready_only_max are prepared, only the
    leading ones whose sort has finished -- the oldest always."""
    take = min(len(events), max_batch)
    if 0 < len(events) <= ready_only_max:
        ready = 1
        while ready < take and events[ready].query():
            ready += 1
        take = ready
    return take


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
    """Latency percentiles and throughput of the completed requests (failed
    ones are counted apart)."""
    ok = [r for r in done if r.error is None]
    lat = np.array([r.latency for r in ok]) * 1000.0 if ok else np.array([math.nan])
    return dict(requests=len(ok), failed=len(done) - len(ok), p50_ms=float(np.percentile(lat, 50)),
                p99_ms=float(np.percentile(lat, 99)), mean_ms=float(lat.mean()), frames_per_s=len(ok) / wall,
                wall_s=wall)
