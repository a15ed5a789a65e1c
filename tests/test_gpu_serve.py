"""The continuous-batching server: every request's image, transmittance and
n_contrib equal a solo gs_render of the same request bit for bit, whatever
batch it was rendered in; a Poisson stream completes with sane latencies."""

import numpy as np
import pytest
import torch

import paper_2509_25626_gb300 as gs
from paper_2509_25626_gb300 import serve as S
from synth import clustered_scene, orbit_camera

pytestmark = pytest.mark.gpu

RES = [(160, 120), (320, 240), (200, 152), (96, 64)]


@pytest.fixture(scope="module")
def server():
    scenes = {name: gs.SceneTensors.from_scene(clustered_scene(n, seed=s), "cuda")
              for name, n, s in (("a", 20000, 11), ("b", 60000, 12), ("c", 120000, 13))}
    srv = S.Server(scenes, max_batch=6, mem_budget=2 << 30)
    for name in scenes:
        for w, h in RES:
            srv.calibrate(name, w, h, [orbit_camera(k, 8, 4.0, w, h) for k in range(8)], margin=2.0)
    return srv


def cam_fn(u, w, h):
    return orbit_camera(u * 8.0, 8, 4.0, w, h)


def solo(srv, req):
    st = srv.scenes[req.scene]
    sp = gs.preprocess(st, req.cam)
    _, vals, ranges, m, _ = gs.sort(sp, st.n, req.cam, 1 << 24)
    return gs.render(sp, vals, ranges, req.cam, req.bg)


def test_batched_results_equal_solo(server):
    reqs = S.poisson_requests(1e9, 1e-6 * 40, list(server.scenes), RES, cam_fn, seed=3)[:40]
    assert len(reqs) >= 20
    done, wall = server.serve(reqs, realtime=False)
    assert len(done) == len(reqs) and server.stats["batches"] < len(reqs)  # requests were batched
    assert server.stats["overflow_or_timeout"] == 0
    for req in done:
        img, T, nc = solo(server, req)
        assert torch.equal(req.image, img) and torch.equal(req.final_T, T) and torch.equal(req.n_contrib, nc)


def test_poisson_stream_completes(server):
    reqs = S.poisson_requests(400.0, 0.5, list(server.scenes), RES, cam_fn, seed=4)
    done, wall = server.serve(reqs, realtime=True)
    st = S.latency_stats(done, wall)
    assert st["requests"] == len(reqs)
    assert all(r.t_done >= r.arrival for r in done)
    assert st["p99_ms"] < 1000.0
    seq_reqs = S.poisson_requests(400.0, 0.5, list(server.scenes), RES, cam_fn, seed=4)
    done2, wall2 = server.serve_sequential(seq_reqs, realtime=True)
    st2 = S.latency_stats(done2, wall2)
    print("batched", st, "sequential", st2)
    for a, b in zip(sorted(done, key=lambda r: r.rid), sorted(done2, key=lambda r: r.rid)):
        assert torch.equal(a.image, b.image)
