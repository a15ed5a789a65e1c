#!/usr/bin/env python3
"""Frames/s of the full 3D Gaussian splatting forward pass (preprocess ->
duplicate keys -> radix sort -> tile ranges -> tile render) on synthetic
scenes, with per-kernel roofline fractions.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gs|reference]

One step renders one frame of the workload (default: 3M Gaussians at
1600x1064, poses cycled over a 20-pose orbit).  Under torchrun each rank
renders its own poses of a replica of the scene (no data-path collective);
the timed region is bracketed by a barrier and a device synchronisation and
the max over ranks is reported.  Rank 0 prints one JSON line.
"""

from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "frames/s at 3M Gaussians 1600x1064 vs roofline; served p50/p99 latency"
FLOP_PER_EVAL = 25  # FP32 work per Gaussian-pixel evaluation of the blend (FMA = 2)
# balanced batch render (gs_render_batch_balanced) settings of the multi-view
# legs: long lists first (heavy_len splats and up), and with splitting
BALANCE_HEAVY = dict(heavy_len=8192, max_heavy_tiles=16384, budget=0, max_split_tiles=0)
BALANCE_SPLIT = dict(heavy_len=8192, max_heavy_tiles=16384, budget=4096, max_split_tiles=4096, max_chunks=32,
                     chunk=1024)


def parse_args():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=1000)
    p.add_argument("--warmup", type=int, default=20)
    p.add_argument("--impl", choices=["gs", "reference"], default="gs")
    p.add_argument("--workload", default="fwd_3m_1600x1064")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-backward", action="store_true")
    p.add_argument("--no-serving", action="store_true")
    p.add_argument("--no-multiview", action="store_true")
    p.add_argument("--no-small", action="store_true", help="skip the 16k-Gaussian 256x256 frame rate")
    p.add_argument("--inflight", type=int, default=3, help="frames in flight on separate streams")
    p.add_argument("--cpu-rows", type=int, default=4, help="tile rows the oracle renders per sampled frame")
    p.add_argument("--profile-frames", type=int, default=0,
                   help="profiler driver: one sizing sort, then this many frames of pose 0 one after another "
                        "(launch order: preprocess + 9 sort kernels, then 11 kernels per frame); no timing")
    p.add_argument("--profile-multiview", type=int, default=0,
                   help="profiler driver: a 2M-Gaussian slab scene (the multi-view recipe at a third of its size), "
                        "two 1920x1080 views preprocessed and sorted, then this many gs_render_batch launches of "
                        "both views; no timing")
    p.add_argument("--profile-split", action="store_true",
                   help="with --profile-multiview: the launches are gs_render_batch_balanced (long lists first, "
                        "heavy tiles split)")
    p.add_argument("--profile-backward", type=int, default=0,
                   help="profiler driver: forward of the 1M-Gaussian 1237x822 backward workload (pose 0), then this "
                        "many backward passes (per pass: gs_render_backward_splats, gs_preprocess_backward); no "
                        "timing")
    return p.parse_args()


def scene_recipe(workload: str) -> dict:
    """The generator settings of the workload's synthetic scene, as the
    bench line states them (the defaults of synth.clustered_scene for the
    clustered workloads)."""
    import inspect
    from synth import clustered_scene
    if workload == "fwd_16k_256":
        return dict(generator="uniform_box_scene", seed=0)
    p = {k: v.default for k, v in inspect.signature(clustered_scene).parameters.items()
         if v.default is not inspect.Parameter.empty}
    seeds = {"fwd_3m_1600x1064": 1, "bwd_1m_1237x822": 3, "slab_6m_3840x2160x8": 5}
    return dict(generator="clustered_scene", seed=seeds.get(workload), n_clusters=p["n_clusters"],
                shell_frac=p["shell_frac"], shell_r=list(p["shell_r"]), ball_r=p["ball_r"],
                axis_std=list(p["axis_std"]), log_scale="centre + t_scale * Student-t(3), clipped",
                log_scale_centre=p["log_scale_centre"], log_scale_t_scale=p["log_scale_t_scale"],
                log_scale_clip=list(p["log_scale_clip"]), opacity_logit_std=p["opacity_std"],
                sh="DC N(0, 0.5), higher bands N(0, 0.05)")


def rank_pose(k: int, world: int, rank: int, n_poses: int) -> int:
    """Pose rendered by `rank` at step k: ranks interleave over the orbit, so
    the N replicas render disjoint poses each step (weak scaling, no data
    exchange)."""
    return (k * world + rank) % n_poses


def max_over_ranks(value: float, world: int, device=None) -> float:
    """The largest `value` over all ranks (the job's time is its slowest
    rank's); identity for a single process."""
    if world <= 1:
        return float(value)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank: int, world: int, max_ms: float) -> float:
    """Units per second of the whole job: every rank's units over the slowest
    rank's time."""
    return units_per_rank * world / (max_ms / 1000.0)


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        return dict(hbm_gbs=float(d["hbm_gbs"]), sm_max_mhz=float(d.get("sm_max_mhz", 2070.0)), src="measured")
    return dict(hbm_gbs=6800.0, sm_max_mhz=2070.0, src="fallback")


class ClockSampler:
    """nvidia-smi clock/throttle samples during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.idx), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"], stdout=self.f,
                                         stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.f.close()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sm.append(float(parts[1]))
                    mx.append(float(parts[2]))
                except ValueError:
                    continue
                for nm, v in zip(names, parts[5:9]):
                    if v.lower().startswith("active"):
                        reasons.add(nm)
        os.unlink(self.path)
        if not sm:
            return None
        return dict(sm_mhz=statistics.median(sm), sm_max_mhz=max(mx), reasons=sorted(reasons), samples=len(sm))


def oracle_frame_sample(scene, cam, rows_tiles: int, threads: int = 0):
    """The FP64 oracle on one frame: full preprocess and sort, then
    ``rows_tiles`` tile rows of the render; returns timings and the
    extrapolated seconds per full frame."""
    from oracle import oracle as O
    O.build_oracle()
    t0 = time.perf_counter()
    pre = O.preprocess(scene, cam)
    t1 = time.perf_counter()
    srt = O.duplicate_sort(pre, cam)
    t2 = time.perf_counter()
    ty = cam.tiles_y
    band0 = max(0, ty // 2 - rows_tiles // 2)
    rows = (16 * band0, min(cam.height, 16 * (band0 + rows_tiles)))
    img = O.render(pre, srt, cam, rows=rows, threads=threads)
    t3 = time.perf_counter()
    frac = (rows[1] - rows[0]) / cam.height
    sec_frame = (t1 - t0) + (t2 - t1) + (t3 - t2) / frac
    cores = os.cpu_count() if (O.has_openmp() and threads <= 0) else max(threads, 1)
    return dict(pre_s=t1 - t0, sort_s=t2 - t1, render_band_s=t3 - t2, band_rows=rows, frac=frac,
                sec_per_frame=sec_frame, cores=cores, m=srt["m"])


_CONFIG1_CODE = r'''
import json, sys, time
sys.path.insert(0, {root!r})
from oracle import oracle as O
from synth import CONFIGS
wl = CONFIGS["fwd_16k_256"]
scene, cam = wl["scene"](), wl["cameras"]()[0]
O.build_oracle()
O.frame(scene, cam)  # warm-up
t = time.perf_counter()
pre, srt, img = O.frame(scene, cam, threads={threads})
dt = time.perf_counter() - t
print(json.dumps(dict(sec_per_frame=dt, evals=int(img["n_eval"].sum()))))
'''


def oracle_config1(threads: int) -> dict:
    """The oracle on the whole 16k-Gaussian 256x256 frame, in a child
    process with OMP_NUM_THREADS = threads (0: all cores)."""
    env = dict(os.environ)
    if threads > 0:
        env["OMP_NUM_THREADS"] = str(threads)
    out = subprocess.run([sys.executable, "-c", _CONFIG1_CODE.format(root=ROOT, threads=threads)], env=env,
                         capture_output=True, text=True, timeout=600)
    r = json.loads(out.stdout.strip().splitlines()[-1])
    r["evals_per_s"] = r["evals"] / r["sec_per_frame"]
    r["threads"] = threads if threads > 0 else os.cpu_count()
    return r


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    # each step is a whole oracle frame sample (seconds): keep the run bounded
    args.steps = min(args.steps, 20)
    args.warmup = min(args.warmup, 3)
    from synth import CONFIGS
    wl = CONFIGS[args.workload]
    scene = wl["scene"]()
    cams = wl["cameras"]()
    times, samples = [], []
    for k in range(args.warmup + args.steps):
        cam = cams[k % len(cams)]
        t = time.perf_counter()
        s = oracle_frame_sample(scene, cam, rows_tiles=1)
        dt = time.perf_counter() - t
        if k >= args.warmup:
            times.append(dt)
            samples.append(s)
    fps = 1.0 / statistics.mean(s["sec_per_frame"] for s in samples)
    cores = samples[0]["cores"]
    line = dict(
        metric=METRIC, value=fps, unit="frames/s", impl="reference", n_gpus=args.gpus, steps=args.steps,
        warmup=args.warmup, ms_per_step=1000.0 * statistics.mean(times), higher_is_better=True,
        scaling="weak", vs_baseline=None, dtype="f64", data="synthetic",
        config=dict(workload=args.workload, gaussians=scene.n, width=cams[0].width, height=cams[0].height,
                    poses=len(cams), scene_recipe=scene_recipe(args.workload)),
        cpu_baseline=dict(value=fps, unit="frames/s", cores=cores, kind="oracle",
                          sample="per step: FP64 oracle preprocess + duplicate/sort of a whole frame and one "
                                 "16-pixel tile row of its render, extrapolated to the full frame"),
        e2e=dict(value=fps, unit="frames/s", h2d_bytes_per_step=0, d2h_bytes_per_step=0),
    )
    print(json.dumps(line), flush=True)
    return 0


def main():
    args = parse_args()
    if args.impl == "reference":
        return run_reference(args)

    import numpy as np
    import torch
    import torch.distributed as dist

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        dist.init_process_group(backend="nccl", device_id=dev)

    def barrier():
        if world > 1:
            dist.barrier()

    if rank == 0:
        from paper_2509_25626_gb300 import build
        build.build()
    barrier()
    import ctypes
    import paper_2509_25626_gb300 as gs
    from paper_2509_25626_gb300 import _lib as L
    from synth import CONFIGS

    if args.profile_multiview > 0:  # fixed launch sequence for ncu captures
        from synth import orbit_camera, slab_scene
        sm_ = slab_scene(2_000_000, seed=5)
        stm = gs.SceneTensors.from_scene(sm_, dev)
        cms = [orbit_camera(k, 8, 4.0, 1920, 1080, arc=math.radians(40.0)) for k in (0, 7)]
        jobs = []
        for cm in cms:
            sp = gs.preprocess(stm, cm)
            _, vals, ranges, _, _ = gs.sort(sp, sm_.n, cm, 1 << 25)
            out = (torch.empty((3, cm.height, cm.width), dtype=torch.float32, device=dev),
                   torch.empty((cm.height, cm.width), dtype=torch.float32, device=dev),
                   torch.empty((cm.height, cm.width), dtype=torch.int32, device=dev))
            jobs.append(gs.BatchJob(sp, vals, ranges, *out, cm.width, cm.height))
        rb = gs.RenderBatch(len(jobs), device=dev)
        rb.set_jobs(jobs)
        bp = gs.BalanceParams(**BALANCE_SPLIT) if args.profile_split else None
        ws = gs.balance_workspace(bp, device=dev) if bp else None
        for _ in range(args.profile_multiview):
            if ws is None:
                rb.launch()
            else:
                rb.launch_balanced(bp, ws)
        torch.cuda.synchronize(dev)
        if rank == 0:
            print(json.dumps({"profile_multiview": args.profile_multiview, "split": bool(args.profile_split),
                              "workload": "slab_2m_1920x1080x2"}))
        return 0

    if args.profile_backward > 0:  # fixed launch sequence for ncu captures
        wb = CONFIGS["bwd_1m_1237x822"]
        sb, cb = wb["scene"](), wb["cameras"]()[0]
        stb = gs.SceneTensors.from_scene(sb, dev)
        sp = gs.preprocess(stb, cb)
        _, vals, ranges, _, _ = gs.sort(sp, sb.n, cb, 8 * sb.n)
        _, Tb, ncb = gs.render(sp, vals, ranges, cb)
        dLb = torch.randn((3, cb.height, cb.width), generator=torch.Generator().manual_seed(0)).to(dev)
        dsplat = torch.empty((sb.n, 12), dtype=torch.float32, device=dev)
        for _ in range(args.profile_backward):
            gs.render_backward_splats(cb, sp, sb.n, vals, ranges, Tb, ncb, dLb, dsplat=dsplat)
            gs.preprocess_backward(stb, cb, sp, dsplat)
        torch.cuda.synchronize(dev)
        if rank == 0:
            print(json.dumps({"profile_backward": args.profile_backward, "workload": "bwd_1m_1237x822"}))
        return 0

    wl = CONFIGS[args.workload]
    scene = wl["scene"]()
    cams = wl["cameras"]()
    P = len(cams)
    st = gs.SceneTensors.from_scene(scene, dev)
    n = scene.n
    W, H = cams[0].width, cams[0].height
    T = gs.num_tiles(cams[0])

    if args.profile_frames > 0:  # fixed launch sequence for ncu captures
        sp = gs.preprocess(st, cams[0])
        _, _, _, m0, _ = gs.sort(sp, n, cams[0], 1 << 24)
        del sp
        rp = gs.Renderer(n, W, H, int(m0 * 1.05) + 4096, dev)
        for _ in range(args.profile_frames):
            rp.frame(st, cams[0])
        torch.cuda.synchronize(dev)
        if rank == 0:
            print(json.dumps({"profile_frames": args.profile_frames, "workload": args.workload, "instances": m0}))
        return 0

    # instance counts per pose (untimed; sizes the key buffers)
    ms = []
    probe_cap = 1 << 24
    for cam in cams:
        sp = gs.preprocess(st, cam)
        while True:
            try:
                _, _, _, m, _ = gs.sort(sp, n, cam, probe_cap)
                break
            except gs.GsError as e:
                if e.code != gs.GS_ERR_CAPACITY:
                    raise
                probe_cap *= 2
        ms.append(m)
        del sp
    torch.cuda.empty_cache()
    m_cap = int(max(ms) * 1.05) + 4096
    r = gs.Renderer(n, W, H, m_cap, dev)

    # evaluations per pose (untimed), the render's work count, and the
    # per-tile block cycles (load balance)
    evals, tile_stats, vis, front, work_stats = [], [], [], [], []
    for cam in cams:
        gs.preprocess(st, cam, r.splats)
        words = r.splats.view(torch.int32)[:n]
        vis.append(int((words[:, 13] > 0).sum().item()))  # tiles_touched > 0
        front.append(int((r.splats[:n, 12] > 0.2).sum().item()))  # in front of the near plane
        gs.sort(r.splats, n, cam, m_cap, r.keys, r.vals, r.ranges, r.workspace, count=False)
        _, _, _, ne, cyc = gs.render_workload(r.splats, r.vals, r.ranges, cam, tile_cycles=True)
        evals.append(int(ne.to(torch.int64).sum().item()))
        tile_stats.append(tile_cycle_stats(cyc))
        work_stats.append(tile_workload_stats(r.ranges, ne, W, H))

    stream = torch.cuda.current_stream(dev)
    pose_of = lambda k: rank_pose(k, world, rank, P)
    E = lambda: torch.cuda.Event(enable_timing=True)

    # frames in flight: frame k runs on stream k % F with its own buffers, so
    # one frame's latency-bound sort and the tail of its render overlap the
    # next frame's work; every frame still runs the whole path
    F = max(1, args.inflight)
    rs = [r] + [gs.Renderer(n, W, H, m_cap, dev) for _ in range(F - 1)]
    streams = [torch.cuda.Stream(dev) for _ in range(F)]

    def run_frames(k0, count, timed):
        fork = E() if timed else torch.cuda.Event()
        fork.record(stream)
        for s_ in streams:
            s_.wait_event(fork)
        for k in range(count):
            i = k % F
            with torch.cuda.stream(streams[i]):
                rs[i].frame(st, cams[pose_of(k0 + k)])
        for s_ in streams:
            j = torch.cuda.Event()
            j.record(s_)
            stream.wait_event(j)

    run_frames(0, args.warmup, False)
    torch.cuda.synchronize(dev)
    start, end = E(), E()
    sampler = ClockSampler(local)
    barrier()
    torch.cuda.synchronize(dev)
    sampler.start()
    start.record(stream)
    run_frames(args.warmup, args.steps, True)
    end.record(stream)
    torch.cuda.synchronize(dev)
    clocks = sampler.stop()
    barrier()
    t_ms = start.elapsed_time(end)
    for r_ in rs:
        assert not r_.instances()[1], "instance capacity overflow during the timed region"
    t_ms = max_over_ranks(t_ms, world, dev)
    fps = whole_job_rate(args.steps, world, t_ms)

    # per-stage times, one frame at a time on one stream (not the headline)
    ks = min(args.steps, 200)
    ev = [[E() for _ in range(4)] for _ in range(ks)]
    s1, e1 = E(), E()
    s1.record(stream)
    for k in range(ks):
        cam = cams[pose_of(args.warmup + k)]
        e = ev[k]
        e[0].record(stream)
        gs.preprocess(st, cam, r.splats)
        e[1].record(stream)
        gs.sort(r.splats, n, cam, m_cap, r.keys, r.vals, r.ranges, r.workspace, count=False)
        e[2].record(stream)
        gs.render(r.splats, r.vals, r.ranges, cam, (0.0, 0.0, 0.0), r.image, r.final_T, r.n_contrib)
        e[3].record(stream)
    e1.record(stream)
    torch.cuda.synchronize(dev)
    serial_fps = ks / (s1.elapsed_time(e1) / 1000.0)
    pre_ms = sum(e[0].elapsed_time(e[1]) for e in ev) / ks
    sort_ms = sum(e[1].elapsed_time(e[2]) for e in ev) / ks
    rend_ms = sum(e[2].elapsed_time(e[3]) for e in ev) / ks
    assert not r.instances()[1], "instance capacity overflow in the per-stage frames"

    # end to end through the public API: scene from pinned host memory each
    # step, image back to pinned host memory; FramePipeline overlaps the
    # upload of frame k+1 with the render of frame k
    e2e = e2e_resident = None
    if not args.no_e2e:
        host = [torch.from_numpy(np.ascontiguousarray(a)).pin_memory() for a in scene.arrays()]
        h2d = sum(h.numel() * h.element_size() for h in host)
        d2h = 3 * H * W * 4
        pipe = gs.FramePipeline(n, W, H, m_cap, dev)
        for k in range(3):
            pipe.result(pipe.submit(host, cams[pose_of(k)]))
        torch.cuda.synchronize(dev)
        barrier()
        s2, e2 = E(), E()
        s2.record(pipe.h2d)
        for k in range(args.steps):
            pipe.submit(host, cams[pose_of(k)])
        e2.record(pipe.d2h)
        torch.cuda.synchronize(dev)
        barrier()
        for t in (pipe.k - 2, pipe.k - 1):
            m_e, over_e = pipe.instances(t)
            assert not over_e, "instance capacity overflow in the end-to-end frames"
        te = max_over_ranks(s2.elapsed_time(e2), world, dev)
        e2e = dict(value=whole_job_rate(args.steps, world, te), unit="frames/s", h2d_bytes_per_step=h2d,
                   d2h_bytes_per_step=d2h, h2d_gbs=h2d * args.steps / (te / 1e3) / 1e9,
                   note="FramePipeline: uploads of frame k+1 overlap the render of frame k")
        del pipe
        # resident scene (a served model): per frame only the camera goes in
        # (kernel parameters) and the image comes back to pinned host memory;
        # frames in flight as for `value`, each image read back on a copy stream
        himgs = [torch.empty((3, H, W), dtype=torch.float32).pin_memory() for _ in range(F)]
        copy_stream = torch.cuda.Stream(dev)
        barrier()
        torch.cuda.synchronize(dev)
        s3, e3 = E(), E()
        s3.record(stream)
        for s_ in streams:
            s_.wait_event(s3)
        done = [None] * F
        for k in range(args.steps):
            i = k % F
            if done[i] is not None:
                streams[i].wait_event(done[i])  # this slot's previous image has been read back
            with torch.cuda.stream(streams[i]):
                rs[i].frame(st, cams[pose_of(k)])
                ev_ = torch.cuda.Event()
                ev_.record(streams[i])
            copy_stream.wait_event(ev_)
            with torch.cuda.stream(copy_stream):
                himgs[i].copy_(rs[i].image, non_blocking=True)
                done[i] = torch.cuda.Event()
                done[i].record(copy_stream)
        stream.wait_stream(copy_stream)
        e3.record(stream)
        torch.cuda.synchronize(dev)
        barrier()
        tr = max_over_ranks(s3.elapsed_time(e3), world, dev)
        e2e_resident = dict(value=whole_job_rate(args.steps, world, tr), unit="frames/s", h2d_bytes_per_step=0,
                            d2h_bytes_per_step=d2h,
                            note="scene resident on the device, camera in as kernel parameters, image out")

    # the render with the optional inverse-depth output (outside the timed frames)
    inv = torch.empty((H, W), dtype=torch.float32, device=dev)
    bgc = (ctypes.c_float * 3)(0.0, 0.0, 0.0)
    reps = max(5, min(args.steps // 10, 50))
    inv_ms = 0.0
    for k in range(reps):
        cam = cams[pose_of(k)]
        r.frame(st, cam)
        c = gs.camera_struct(cam)
        a, b = E(), E()
        a.record(stream)
        L.check(L.lib().gs_render_ex(ctypes.c_void_p(r.splats.data_ptr()), ctypes.c_void_p(r.vals.data_ptr()),
                                     ctypes.c_void_p(r.ranges.data_ptr()), ctypes.byref(c), bgc,
                                     ctypes.c_void_p(r.image.data_ptr()), ctypes.c_void_p(r.final_T.data_ptr()),
                                     ctypes.c_void_p(r.n_contrib.data_ptr()), ctypes.c_void_p(inv.data_ptr()), None,
                                     None, ctypes.c_void_p(stream.cuda_stream)), "gs_render_ex")
        b.record(stream)
        torch.cuda.synchronize(dev)
        inv_ms += a.elapsed_time(b) / reps
    # the contribution-aware (Seele-style) render on the same frames
    ca_ms = 0.0
    for k in range(reps):
        cam = cams[pose_of(k)]
        r.frame(st, cam)
        a, b = E(), E()
        a.record(stream)
        gs.render_contrib(r.splats, r.vals, r.ranges, cam, (0.0, 0.0, 0.0), r.image, r.final_T, r.n_contrib,
                          stream=stream)
        b.record(stream)
        torch.cuda.synchronize(dev)
        ca_ms += a.elapsed_time(b) / reps

    # roofline of the dominant kernel (the render: FP32 issue bound)
    peaks = measured_peaks()
    props = torch.cuda.get_device_properties(dev)
    sms = props.multi_processor_count
    fp32_peak = sms * 128 * 2 * peaks["sm_max_mhz"] * 1e6 / 1e12  # TFLOP/s at the max SM clock
    used = [pose_of(args.warmup + k) for k in range(ks)]
    evals_mean = statistics.mean(evals[p] for p in used)
    ms_mean = statistics.mean(ms[p] for p in used)
    render_tflops = evals_mean * FLOP_PER_EVAL / (rend_ms / 1000.0) / 1e12
    # preprocess bytes: every Gaussian's mean; scales and rotation of those
    # in front of the near plane; opacity and SH of the visible ones (culled
    # Gaussians need neither); out, the whole record of a visible Gaussian,
    # the last 32 bytes of a culled one's, and every dense sort input
    front_mean = statistics.mean(front[p] for p in used)
    vis_mean = statistics.mean(vis[p] for p in used)
    pre_bytes = n * 12 + front_mean * 28 + vis_mean * (4 + 192) + vis_mean * 64 + (n - vis_mean) * 32 + n * 16
    pre_gbs = pre_bytes / (pre_ms / 1000.0) / 1e9
    traffic = None
    try:
        with open(os.path.join(ROOT, "profiles", "render_traffic.json")) as f:
            tr = json.load(f)
        if tr.get("workload") == args.workload and tr.get("kernel_source_sha") == kernel_sha("render.cu", "common.cuh"):
            traffic = tr.get("dram_bytes_per_launch")
    except (OSError, ValueError):
        pass
    roofline = dict(bound="alu", achieved=render_tflops, peak=fp32_peak, unit="TFLOP/s",
                    frac=render_tflops / fp32_peak, traffic=traffic,
                    kernel="render", work=f"{evals_mean:.4g} Gaussian-pixel evaluations x {FLOP_PER_EVAL} FLOP",
                    peak_src=f"{sms} SMs x 128 FP32 lanes x 2 x {peaks['sm_max_mhz']:.0f} MHz")
    if clocks and clocks.get("sm_mhz"):
        roofline["frac_at_sampled_clock"] = render_tflops / (sms * 256 * clocks["sm_mhz"] * 1e6 / 1e12)
    kernels = dict(
        preprocess=dict(ms=pre_ms, bytes=pre_bytes, gbs=pre_gbs, frac_hbm=pre_gbs / peaks["hbm_gbs"]),
        sort=dict(ms=sort_ms, instances=ms_mean),  # bytes and fraction below, with the frame roofline
        render_invdepth=dict(ms=inv_ms, tflops=evals_mean * FLOP_PER_EVAL / (inv_ms / 1000.0) / 1e12,
                             frac=evals_mean * FLOP_PER_EVAL / (inv_ms / 1000.0) / 1e12 / fp32_peak,
                             note="render with the optional inverse-depth output, same poses; work as the "
                                  "render's (the depth channel's FMA not counted)"),
        render_contrib=dict(ms=ca_ms, tflops=evals_mean * FLOP_PER_EVAL / (ca_ms / 1000.0) / 1e12,
                            frac=evals_mean * FLOP_PER_EVAL / (ca_ms / 1000.0) / 1e12 / fp32_peak,
                            note="contribution-aware (Seele-style) render: per-warp vote masks, then the blend of "
                                 "the masked splats; the same outputs, same poses, work counted as the render's"),
        render=dict(ms=rend_ms, evals=evals_mean, evals_per_s=evals_mean / (rend_ms / 1000.0), tflops=render_tflops,
                    tile_cycles={k: statistics.mean(t[k] for t in tile_stats) for k in tile_stats[0]},
                    workload={k: statistics.mean(t[k] for t in work_stats) for k in work_stats[0]}),
    )
    # kernels per frame: preprocess; compact, 4 depth radix passes, offsets,
    # duplicate fused with the first tile pass, one more pass per further
    # byte of the tile key (a byte of tx, then of ty), ranges; render
    tiles_x, tiles_y = (W + 15) // 16, (H + 15) // 16
    key_bytes = lambda c: 0 if c <= 1 else (1 if c <= 256 else 2)
    tile_passes = max(1, key_bytes(tiles_x)) + key_bytes(tiles_y)
    launches_per_frame = 1 + (1 + 4 + 1 + tile_passes + 1) + 1

    # frame roofline: each step's floor (HBM bytes / measured HBM for the
    # preprocess and the sort, the FP32 issue floor for the render) summed,
    # against the measured frame time (frames one at a time)
    nvis = vis_mean
    sort_bytes = (n * 16 + nvis * 12                     # compaction: sort inputs in; keys, ids, depth out
                  + 4 * nvis * 16                        # four depth passes: (key, id) in and out
                  + nvis * 12                            # offsets: ids, rectangles, offsets
                  + ms_mean * 8                          # duplicate + first tile pass: (tile, id) out
                  + ms_mean * 20                         # last tile pass: 8 B in, 12 B out
                  + T * 8)                               # ranges
    floors = dict(preprocess_ms=pre_bytes / (peaks["hbm_gbs"] * 1e6),
                  sort_ms=sort_bytes / (peaks["hbm_gbs"] * 1e6),
                  render_ms=evals_mean * FLOP_PER_EVAL / (fp32_peak * 1e9))
    kernels["sort"].update(bytes=sort_bytes, gbs=sort_bytes / (sort_ms / 1000.0) / 1e9,
                           frac_hbm=sort_bytes / (sort_ms / 1000.0) / 1e9 / peaks["hbm_gbs"],
                           bound="latency and issue; fraction of its algorithmic bytes at HBM speed")
    frame_roofline = dict(floor_ms=sum(floors.values()), frame_ms=1000.0 / serial_fps,
                          frac=sum(floors.values()) / (1000.0 / serial_fps), **floors,
                          sort_bytes=sort_bytes)

    serving = None
    if rank == 0 and not args.no_serving:
        serving = measure_serving(gs, dev)

    small = None
    if rank == 0 and not args.no_small:
        small = measure_small_config(gs, dev)
    multiview = None
    if rank == 0 and not args.no_multiview:
        multiview = measure_multiview(gs, dev)

    backward = None
    if not args.no_backward:
        backward = measure_backward(gs, dev, steps=max(3, min(args.steps // 20, 50)), warmup=3)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        s = oracle_frame_sample(scene, cams[used[0]], rows_tiles=args.cpu_rows)
        cpu = dict(value=1.0 / s["sec_per_frame"], unit="frames/s", cores=s["cores"], kind="oracle",
                   sample=f"one frame (pose {used[0]}): FP64 oracle preprocess ({s['pre_s']:.2f} s) and "
                          f"duplicate/sort ({s['sort_s']:.2f} s) in full, render of pixel rows {s['band_rows']} "
                          f"({s['render_band_s']:.2f} s) extrapolated to the whole image")
        try:
            cpu["config_fwd_16k_256"] = dict(one_thread=oracle_config1(1), all_cores=oracle_config1(0))
        except (subprocess.SubprocessError, ValueError, IndexError, KeyError) as e:
            cpu["config_fwd_16k_256"] = dict(error=str(e)[:200])

    if rank == 0:
        line = dict(
            metric=METRIC, value=fps, unit="frames/s", n_gpus=world, steps=args.steps, warmup=args.warmup,
            ms_per_step=t_ms / args.steps, higher_is_better=True, scaling="weak", vs_baseline=None,
            dtype="f32", data="synthetic",
            config=dict(workload=args.workload, gaussians=n, width=W, height=H, poses=P, tiles=T,
                        instances_mean=ms_mean, visible_pose0=vis[0], evals_mean=evals_mean,
                        m_cap=m_cap, parallelism=f"replicas{world}", frames_in_flight=F,
                        serial_frames_per_s=serial_fps, scene_recipe=scene_recipe(args.workload),
                        l2="inputs larger than L2: the 708 MB scene is re-read from HBM every frame"),
            roofline=roofline, frame_roofline=frame_roofline, kernels=kernels, cpu_baseline=cpu, e2e=e2e,
            e2e_resident_scene=e2e_resident,
            serving=serving, multiview=multiview, small_config=small,
            backward=backward,
            gpu_launches=launches_per_frame * args.steps, clocks=clocks,
            peaks_src=peaks["src"],
        )
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


def tile_workload_stats(ranges, n_eval, width: int, height: int) -> dict:
    """The per-tile and per-thread workload the paper characterises (Table
    III): Gaussians per tile (list length) over every tile, mean and
    variance; and, per pixel of a non-empty tile, the fraction of its tile's
    list it evaluates before stopping, mean and variance."""
    import torch
    r = ranges.to(torch.int64)
    lens = (r[:, 1] - r[:, 0]).to(torch.float64)
    tiles_x = (width + 15) // 16
    py = torch.arange(height, device=lens.device).view(-1, 1) // 16
    px = torch.arange(width, device=lens.device).view(1, -1) // 16
    per_px = lens[(py * tiles_x + px).reshape(-1)].reshape(height, width)
    ok = per_px > 0
    frac = n_eval.to(torch.float64)[ok] / per_px[ok]
    return dict(gaussians_per_tile_mean=float(lens.mean()), gaussians_per_tile_var=float(lens.var(unbiased=False)),
                evaluated_fraction_mean=float(frac.mean()), evaluated_fraction_var=float(frac.var(unbiased=False)))


def tile_cycle_stats(cyc) -> dict:
    """Per-tile block cycles (gs_render_workload): mean, p99, max, max/mean."""
    import torch
    c = cyc.reshape(-1).to(torch.float64)
    mean = float(c.mean())
    return dict(mean=mean, p99=float(torch.quantile(c, 0.99)), max=float(c.max()),
                max_over_mean=float(c.max()) / max(mean, 1.0), sum=float(c.sum()))


def measure_serving(gs, dev, rates=(200.0, 800.0, 1600.0, 2400.0), duration: float = 1.0):
    """Continuous-batching server on three resident scenes (0.5M, 2M, 5M
    Gaussians, clustered like the 3M workload), Poisson arrivals at each
    offered rate, each request a random orbit pose at a resolution drawn
    from {640x480, 1280x720, 1600x1064, 1920x1080}.  Per rate: latency
    percentiles and delivered frames/s of the batched server and of
    one-request-at-a-time rendering on the same slots and captured graphs;
    plus both at saturation (all requests present at t = 0)."""
    from paper_2509_25626_gb300 import serve as S
    from synth import clustered_scene, orbit_camera
    specs = (("s0.5m", 500_000, 41), ("s2m", 2_000_000, 42), ("s5m", 5_000_000, 43))
    scenes = {name: gs.SceneTensors.from_scene(clustered_scene(n, seed=sd), dev) for name, n, sd in specs}
    res = [(640, 480), (1280, 720), (1600, 1064), (1920, 1080)]
    srv = S.Server(scenes, res, max_batch=16, mem_budget=96 << 30, device=dev, slots_per_scene=12)
    for name in scenes:
        for w, h in res:
            srv.calibrate(name, w, h, [orbit_camera(k, 6, 4.0, w, h) for k in range(6)])
    cam_fn = lambda u, w, h: orbit_camera(u * 20.0, 20, 4.0, w, h)
    srv.serve(S.poisson_requests(rates[0], 0.3, list(scenes), res, cam_fn, seed=97), realtime=True)  # warm-up
    srv.serve_sequential(S.poisson_requests(rates[0], 0.1, list(scenes), res, cam_fn, seed=96), realtime=True)
    out = {"rates": {}}
    for rate in rates:
        row = {}
        dur = max(duration, 500.0 / rate)  # at least ~500 requests per rate, so that p99 is not the maximum
        for mode in ("batched", "sequential"):
            reqs = S.poisson_requests(rate, dur, list(scenes), res, cam_fn, seed=99)
            fn = srv.serve if mode == "batched" else srv.serve_sequential
            done, wall = fn(reqs, realtime=True)
            row[mode] = S.latency_stats(done, wall)
            row[mode]["offered_per_s"] = len(reqs) / dur
        out["rates"][f"{int(rate)}"] = row
    for mode in ("batched", "sequential"):
        sat = S.poisson_requests(rates[-1], duration, list(scenes), res, cam_fn, seed=100)
        for r in sat:
            r.arrival = 0.0
        fn = srv.serve if mode == "batched" else srv.serve_sequential
        done, wall = fn(sat, realtime=False)
        out[f"saturated_{mode}_frames_per_s"] = S.latency_stats(done, wall)["frames_per_s"]
    out.update(workload="serve_3scenes_poisson", duration_s=duration,
               scenes={name: n for name, n, _ in specs}, resolutions=[f"{w}x{h}" for w, h in res],
               slots={k: int(v) for k, v in srv.stats.items() if k.startswith("slots_")},
               batches=int(srv.stats["batches"]), failed=int(srv.stats["failed"]))
    return out


def measure_small_config(gs, dev, frames: int = 500):
    """The 16,384-Gaussian 256x256 frame (its one pose): whole frames
    (preprocess, sort, render) one after another on one stream, CUDA events
    around them.  Its 3.9 MB scene stays in L2 between frames (not flushed):
    a frame this small is bound by launch and latency, not by HBM."""
    import torch
    from synth import CONFIGS
    wl = CONFIGS["fwd_16k_256"]
    scene, cam = wl["scene"](), wl["cameras"]()[0]
    st = gs.SceneTensors.from_scene(scene, dev)
    sp = gs.preprocess(st, cam)
    _, _, _, m, _ = gs.sort(sp, scene.n, cam, 1 << 22)
    del sp
    r = gs.Renderer(scene.n, cam.width, cam.height, int(m * 1.05) + 4096, dev)
    for _ in range(10):
        r.frame(st, cam)
    stream = torch.cuda.current_stream(dev)
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize(dev)
    a.record(stream)
    for _ in range(frames):
        r.frame(st, cam)
    b.record(stream)
    torch.cuda.synchronize(dev)
    ms = a.elapsed_time(b) / frames
    ne = gs.render_workload(r.splats, r.vals, r.ranges, cam)[3]
    evals = int(ne.to(torch.int64).sum().item())
    return dict(workload="fwd_16k_256", gaussians=scene.n, width=cam.width, height=cam.height, frames=frames,
                instances=int(m), ms_per_frame=ms, frames_per_s=1000.0 / ms, evals=evals,
                evals_per_s=evals / (ms / 1000.0), l2="scene resident in L2 between frames (3.9 MB)")


def measure_multiview(gs, dev, steps: int = 5):
    """Load-imbalance workload: 6M Gaussians, half packed in an occluding
    slab, 8 views at 3840x2160.  Per step: the 8 views' preprocess and sort
    (one stream per view), then their renders in ONE persistent launch
    (gs_render_batch); compared with the same renders as 8 separate
    gs_render launches."""
    import ctypes
    import torch
    from paper_2509_25626_gb300 import _lib as L
    from paper_2509_25626_gb300 import serve as S
    from synth import CONFIGS
    wl = CONFIGS["slab_6m_3840x2160x8"]
    scene = wl["scene"]()
    cams = wl["cameras"]()
    st = gs.SceneTensors.from_scene(scene, dev)
    ms = []
    for cam in cams:
        sp = gs.preprocess(st, cam)
        _, _, _, m, _ = gs.sort(sp, st.n, cam, 1 << 27)
        ms.append(m)
        del sp
    rs = [gs.Renderer(st.n, cam.width, cam.height, int(max(ms) * 1.05) + 4096, dev) for cam in cams]
    rb = gs.RenderBatch(len(cams), device=dev)
    tiles = rb.set_jobs([gs.BatchJob(r.splats, r.vals, r.ranges, r.image, r.final_T, r.n_contrib, c.width, c.height)
                         for r, c in zip(rs, cams)])
    bal = {k: gs.BalanceParams(**v) for k, v in (("heavy", BALANCE_HEAVY), ("split", BALANCE_SPLIT))}
    bal_ws = {k: gs.balance_workspace(v, device=dev) for k, v in bal.items()}
    stream = torch.cuda.current_stream(dev)

    # each view's preprocess and sort on a stream of its own (the views are
    # independent and their sorts are latency-bound), forked from and joined
    # to the timing stream
    view_streams = [torch.cuda.Stream(dev) for _ in cams]

    def front():
        fork = torch.cuda.Event()
        fork.record(stream)
        for vs, r, cam in zip(view_streams, rs, cams):
            vs.wait_event(fork)
            gs.preprocess(st, cam, r.splats, stream=vs)
            gs.sort(r.splats, st.n, cam, r.m_cap, r.keys, r.vals, r.ranges, r.workspace, count=False, stream=vs)
        for vs in view_streams:
            join = torch.cuda.Event()
            join.record(vs)
            stream.wait_event(join)

    def batched():
        rb.launch()

    def batched_heavy():
        rb.launch_balanced(bal["heavy"], bal_ws["heavy"])

    def batched_split():
        rb.launch_balanced(bal["split"], bal_ws["split"])

    def separate():
        for r, cam in zip(rs, cams):
            gs.render(r.splats, r.vals, r.ranges, cam, (0.0, 0.0, 0.0), r.image, r.final_T, r.n_contrib)

    E = lambda: torch.cuda.Event(enable_timing=True)
    res = {}
    for name, fn in (("batched", batched), ("batched_long_first", batched_heavy), ("batched_split", batched_split),
                     ("separate", separate)):
        front()
        fn()
        torch.cuda.synchronize(dev)
        t_front = t_render = 0.0
        for _ in range(steps):
            a, b, c = E(), E(), E()
            a.record(stream)
            front()
            b.record(stream)
            fn()
            c.record(stream)
            torch.cuda.synchronize(dev)
            t_front += a.elapsed_time(b)
            t_render += b.elapsed_time(c)
        res[name] = dict(render_ms=t_render / steps, preprocess_sort_ms=t_front / steps,
                         views_per_s=len(cams) * 1000.0 / ((t_front + t_render) / steps))

    # pipelined: each view's preprocess, sort and render on its own stream,
    # so one view's render overlaps the others' sorts (whole step timed)
    def pipelined():
        fork = torch.cuda.Event()
        fork.record(stream)
        for vs, r, cam in zip(view_streams, rs, cams):
            vs.wait_event(fork)
            gs.preprocess(st, cam, r.splats, stream=vs)
            gs.sort(r.splats, st.n, cam, r.m_cap, r.keys, r.vals, r.ranges, r.workspace, count=False, stream=vs)
            gs.render(r.splats, r.vals, r.ranges, cam, (0.0, 0.0, 0.0), r.image, r.final_T, r.n_contrib, stream=vs)
        for vs in view_streams:
            join = torch.cuda.Event()
            join.record(vs)
            stream.wait_event(join)

    pipelined()
    torch.cuda.synchronize(dev)
    a, b = E(), E()
    a.record(stream)
    for _ in range(steps):
        pipelined()
    b.record(stream)
    torch.cuda.synchronize(dev)
    step_ms = a.elapsed_time(b) / steps
    pipe = dict(step_ms=step_ms, views_per_s=len(cams) * 1000.0 / step_ms)
    lens, cycs, evals = [], [], 0
    for r, cam in zip(rs, cams):
        rg = r.ranges.to(torch.int64)
        lens.append((rg[:, 1] - rg[:, 0]).cpu())
        wl_out = gs.render_workload(r.splats, r.vals, r.ranges, cam, tile_cycles=True)
        evals += int(wl_out[3].to(torch.int64).sum().item())
        cycs.append(wl_out[4].reshape(-1).cpu())
    lens = torch.cat(lens).float()
    tc = tile_cycle_stats(torch.cat(cycs))
    # the renders' roofline: Gaussian-pixel evaluations of the 8 views (the
    # untimed workload render above) x FLOP_PER_EVAL over the FP32 issue peak
    peaks = measured_peaks()
    fp32_peak = torch.cuda.get_device_properties(dev).multi_processor_count * 256 * peaks["sm_max_mhz"] * 1e6 / 1e12
    for v in res.values():
        v["tflops"] = evals * FLOP_PER_EVAL / (v["render_ms"] / 1000.0) / 1e12
        v["frac"] = v["tflops"] / fp32_peak
    res["evals"] = evals
    res["pipelined"] = pipe
    res["balance_params"] = dict(long_first=BALANCE_HEAVY, split=BALANCE_SPLIT,
                                 long_tiles=int(bal_ws["split"][8:12].view(torch.int32).item()),
                                 split_tiles=int(bal_ws["split"][:4].view(torch.int32).item()))
    res["slab_2m_1920x1080x2"] = measure_split_small(gs, dev, steps=max(steps, 10))
    return dict(workload="slab_6m_3840x2160x8", gaussians=st.n, views=len(cams), tiles=int(tiles),
                instances_mean=float(sum(ms) / len(ms)), tile_list_mean=float(lens.mean()),
                tile_list_max=int(lens.max()), tile_list_var=float(lens.var()), tile_cycles=tc, **res)


def measure_split_small(gs, dev, steps: int = 10):
    """The load-imbalance recipe at a third of its size and a quarter of its
    pixels (2M Gaussians, two 1920x1080 views), where a few slab-edge tiles
    dominate the batch launch: gs_render_batch against gs_render_batch_split
    (render only, the same sorted inputs)."""
    import torch
    from synth import orbit_camera, slab_scene
    sc = slab_scene(2_000_000, seed=5)
    st = gs.SceneTensors.from_scene(sc, dev)
    cams = [orbit_camera(k, 8, 4.0, 1920, 1080, arc=math.radians(40.0)) for k in (0, 7)]
    jobs = []
    for cam in cams:
        sp = gs.preprocess(st, cam)
        _, vals, ranges, _, _ = gs.sort(sp, sc.n, cam, 1 << 25)
        out = (torch.empty((3, cam.height, cam.width), dtype=torch.float32, device=dev),
               torch.empty((cam.height, cam.width), dtype=torch.float32, device=dev),
               torch.empty((cam.height, cam.width), dtype=torch.int32, device=dev))
        jobs.append(gs.BatchJob(sp, vals, ranges, *out, cam.width, cam.height))
    rb = gs.RenderBatch(len(jobs), device=dev)
    rb.set_jobs(jobs)
    bal = {k: gs.BalanceParams(**v) for k, v in (("heavy", BALANCE_HEAVY), ("split", BALANCE_SPLIT))}
    bal_ws = {k: gs.balance_workspace(v, device=dev) for k, v in bal.items()}
    stream = torch.cuda.current_stream(dev)
    E = lambda: torch.cuda.Event(enable_timing=True)
    out = {}
    for name, fn in (("batched", lambda: rb.launch()),
                     ("batched_long_first", lambda: rb.launch_balanced(bal["heavy"], bal_ws["heavy"])),
                     ("batched_split", lambda: rb.launch_balanced(bal["split"], bal_ws["split"]))):
        for _ in range(3):
            fn()
        torch.cuda.synchronize(dev)
        a, b = E(), E()
        a.record(stream)
        for _ in range(steps):
            fn()
        b.record(stream)
        torch.cuda.synchronize(dev)
        out[name] = dict(render_ms=a.elapsed_time(b) / steps)
    out["long_tiles"] = int(bal_ws["split"][8:12].view(torch.int32).item())
    out["split_tiles"] = int(bal_ws["split"][:4].view(torch.int32).item())
    out["speedup_long_first"] = out["batched"]["render_ms"] / out["batched_long_first"]["render_ms"]
    out["speedup_split"] = out["batched"]["render_ms"] / out["batched_split"]["render_ms"]
    return out


def measure_backward(gs, dev, steps: int, warmup: int):
    """Forward + backward of the 1M-Gaussian 1237x822 workload (orbit poses,
    upstream gradient N(0, 1) per pixel and channel): ms per training step."""
    import numpy as np
    import torch
    from synth import CONFIGS
    wl = CONFIGS["bwd_1m_1237x822"]
    scene = wl["scene"]()
    cams = wl["cameras"]()
    params = [torch.from_numpy(np.ascontiguousarray(a)).to(dev).requires_grad_(True) for a in scene.arrays()]
    g = torch.Generator(device=dev).manual_seed(0)
    dL = torch.randn((3, cams[0].height, cams[0].width), generator=g, device=dev)
    def step(k):
        for p_ in params:  # as zero_grad(set_to_none=True): the new gradients are assigned, not added
            p_.grad = None
        img = gs.rasterize(*params, cams[k % len(cams)], (0.0, 0.0, 0.0), 3)
        img.backward(dL)
    for k in range(warmup):
        step(k)
    torch.cuda.synchronize(dev)
    s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    s.record()
    for k in range(steps):
        step(k)
    e.record()
    torch.cuda.synchronize(dev)
    ms = s.elapsed_time(e) / steps

    # the backward's two kernels timed apart on the forward's outputs, with
    # their roofline fractions: the backward render against the FP32 issue
    # peak (work: the evaluations it walks, sum of n_contrib over pixels,
    # x the forward's 25 FLOP of recomputation -- a lower bound, the gradient
    # terms of blended evaluations come on top); the preprocess backward
    # against HBM (bytes it must move: the tiles word and the 236 B of
    # gradients of every Gaussian, plus the 2D gradients (48 B) and the
    # parameters (236 B) of the visible ones)
    st = gs.SceneTensors.from_scene(scene, dev)
    n = scene.n
    dsplat = torch.empty((n, 12), dtype=torch.float32, device=dev)
    grads = {k: torch.empty_like(getattr(st, k)) for k in ("means", "log_scales", "quats", "opacity_logits", "sh")}
    peaks = measured_peaks()
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    fp32_peak = sms * 128 * 2 * peaks["sm_max_mhz"] * 1e6 / 1e12
    E = lambda: torch.cuda.Event(enable_timing=True)
    t_rb = t_pb = 0.0
    evals = vis = 0
    reps = len(cams)
    for k in range(reps + 1):  # the first pass warms up
        cam = cams[k % len(cams)]
        sp = gs.preprocess(st, cam)
        _, vals, ranges, _, _ = gs.sort(sp, n, cam, 8 * n)
        _, T, nc = gs.render(sp, vals, ranges, cam)
        a, b, c = E(), E(), E()
        a.record()
        gs.render_backward_splats(cam, sp, n, vals, ranges, T, nc, dL, dsplat=dsplat)
        b.record()
        gs.preprocess_backward(st, cam, sp, dsplat, grads)
        c.record()
        torch.cuda.synchronize(dev)
        if k > 0:
            t_rb += a.elapsed_time(b) / reps
            t_pb += b.elapsed_time(c) / reps
            evals += int(nc.to(torch.int64).sum().item())
            vis += int((sp[:n].view(torch.int32)[:, 13] > 0).sum().item())
    evals /= reps
    vis /= reps
    rb_tflops = evals * FLOP_PER_EVAL / (t_rb / 1000.0) / 1e12
    pb_bytes = n * (4 + 236) + vis * (48 + 236)
    pb_gbs = pb_bytes / (t_pb / 1000.0) / 1e9
    kernels = dict(
        render_backward=dict(ms=t_rb, evals=evals, tflops=rb_tflops, frac=rb_tflops / fp32_peak, bound="alu",
                             work=f"{evals:.4g} evaluations (sum of n_contrib) x {FLOP_PER_EVAL} FLOP, lower bound"),
        preprocess_backward=dict(ms=t_pb, bytes=pb_bytes, gbs=pb_gbs, frac_hbm=pb_gbs / peaks["hbm_gbs"],
                                 bound="hbm"))
    return dict(workload="bwd_1m_1237x822", gaussians=scene.n, width=cams[0].width, height=cams[0].height,
                steps=steps, ms_per_step=ms, steps_per_s=1000.0 / ms, kernels=kernels,
                note="forward + backward through gs.rasterize (one host sync per forward for the sort's M); "
                     "parameter gradients set to None before each step, as zero_grad does")


def kernel_sha(*names: str) -> str:
    """First 16 hex digits of the SHA-256 of the named csrc files, in order."""
    import hashlib
    h = hashlib.sha256()
    for name in names:
        with open(os.path.join(ROOT, "paper_2509_25626_gb300", "csrc", name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


if __name__ == "__main__":
    sys.exit(main())
