"""The continuous-batching server: every request's image, transmittance and
n_contrib equal a solo gs_render of the same request bit for bit, whatever
batch and slot it was rendered in, through the captured preprocess + sort
graphs (the pose entering through the slot's device camera block) or
without them; a Poisson stream completes with sane latencies; a request
whose instances overflow its slot is returned as failed, not truncated."""

import pytest
import torch

import paper_2509_25626_gb300 as gs
from paper_2509_25626_gb300 import serve as S
from synth import clustered_scene, orbit_camera

pytestmark = pytest.mark.gpu

RES = [(160, 120), (320, 240), (200, 152), (96, 64)]


def _scenes():
    return {name: gs.SceneTensors.from_scene(clustered_scene(n, seed=s), "cuda")
            for name, n, s in (("a", 20000, 11), ("b", 60000, 12), ("c", 120000, 13))}


def _server(scenes, **kw):
    srv = S.Server(scenes, RES, max_batch=6, mem_budget=2 << 30, slots_per_scene=4, **kw)
    for name in scenes:
        for w, h in RES:
            srv.calibrate(name, w, h, [orbit_camera(k, 8, 4.0, w, h) for k in range(8)], margin=2.0)
    return srv


@pytest.fixture(scope="module")
def scenes():
    return _scenes()


@pytest.fixture(scope="module")
def server(scenes):
    return _server(scenes)


def cam_fn(u, w, h):
    return orbit_camera(u * 8.0, 8, 4.0, w, h)


def solo(scenes, req):
    st = scenes[req.scene]
    sp = gs.preprocess(st, req.cam)
    _, vals, ranges, m, _ = gs.sort(sp, st.n, req.cam, 1 << 24)
    return gs.render(sp, vals, ranges, req.cam, req.bg)


def test_batched_results_equal_solo(server, scenes):
    reqs = S.poisson_requests(1e9, 1e-6 * 40, list(scenes), RES, cam_fn, seed=3)[:40]
    assert len(reqs) >= 20
    done, wall = server.serve(reqs, realtime=False)
    assert len(done) == len(reqs) and server.stats["batches"] < len(reqs)  # requests were batched
    assert server.stats["failed"] == 0 and server.graph is not None
    for req in done:
        assert req.error is None
        img, T, nc = solo(scenes, req)
        assert torch.equal(req.image, img) and torch.equal(req.final_T, T) and torch.equal(req.n_contrib, nc)


def test_without_graphs_equal(scenes):
    """The same requests without the captured graphs (direct calls)."""
    srv = _server(scenes, use_graph=False)
    reqs = S.poisson_requests(1e9, 1e-6 * 20, list(scenes), RES, cam_fn, seed=5)[:20]
    done, _ = srv.serve(reqs, realtime=False)
    for req in done:
        img, T, nc = solo(scenes, req)
        assert torch.equal(req.image, img) and torch.equal(req.final_T, T) and torch.equal(req.n_contrib, nc)


def test_poisson_stream_completes(server, scenes):
    reqs = S.poisson_requests(400.0, 0.5, list(scenes), RES, cam_fn, seed=4)
    done, wall = server.serve(reqs, realtime=True)
    st = S.latency_stats(done, wall)
    assert st["requests"] == len(reqs) and st["failed"] == 0
    assert all(r.t_done >= r.arrival for r in done)
    assert st["p99_ms"] < 1000.0
    seq_reqs = S.poisson_requests(400.0, 0.5, list(scenes), RES, cam_fn, seed=4)
    done2, wall2 = server.serve_sequential(seq_reqs, realtime=True)
    st2 = S.latency_stats(done2, wall2)
    print("batched", st, "sequential", st2)
    for a, b in zip(sorted(done, key=lambda r: r.rid), sorted(done2, key=lambda r: r.rid)):
        assert torch.equal(a.image, b.image)


def test_overflowing_request_fails_cleanly(scenes):
    """Scene "c"'s slots get a capacity far below its instance count: its
    requests come back failed (error "capacity", no image, the true instance
    count reported) and stay out of the latency statistics; the other
    scenes' requests in the same batches are exact."""
    srv = _server(scenes)
    for w, h in RES:
        srv.m_caps[("c", w, h)] = 512
    reqs = S.poisson_requests(1e9, 1e-6 * 30, list(scenes), RES, cam_fn, seed=6)[:30]
    assert any(r.scene == "c" for r in reqs) and any(r.scene != "c" for r in reqs)
    done, wall = srv.serve(reqs, realtime=False)
    st = S.latency_stats(done, wall)
    n_c = sum(r.scene == "c" for r in reqs)
    assert st["failed"] == n_c == srv.stats["failed"] and st["requests"] == len(reqs) - n_c
    for req in done:
        if req.scene == "c":
            assert req.error == "capacity" and req.image is None and req.instances > 512
        else:
            assert req.error is None
            img, T, nc = solo(scenes, req)
            assert torch.equal(req.image, img) and torch.equal(req.n_contrib, nc)
