"""FramePipeline (double-buffered host-to-host frames) vs Renderer.frame:
the same images, bit for bit, for a sequence of different scenes and poses,
whichever slot a frame lands in."""

import numpy as np
import pytest
import torch

import paper_2509_25626_gb300 as gs
from synth import clustered_scene, orbit_camera

pytestmark = pytest.mark.gpu


def test_pipeline_equals_renderer_frames():
    base = clustered_scene(30000, seed=4)
    cams = [orbit_camera(k, 20, 4.0, 320, 240) for k in (0, 3, 7, 11, 15)]
    rng = np.random.default_rng(0)
    scenes = []
    for k in range(len(cams)):  # each frame its own scene: perturbed means and colours
        arrs = [a.copy() for a in base.arrays()]
        arrs[0] += rng.normal(0, 0.01, size=arrs[0].shape).astype(np.float32)
        arrs[4][:, 0, :] += rng.normal(0, 0.1, size=arrs[4][:, 0, :].shape).astype(np.float32)
        scenes.append(arrs)
    r = gs.Renderer(base.n, 320, 240, 4_000_000)
    refs = []
    for arrs, cam in zip(scenes, cams):
        st = gs.SceneTensors.from_arrays(*arrs)
        img, _, _ = r.frame(st, cam, (0.1, 0.2, 0.3))
        refs.append(img.cpu().clone())
    pipe = gs.FramePipeline(base.n, 320, 240, 4_000_000)
    hosts = [[torch.from_numpy(np.ascontiguousarray(a)).pin_memory() for a in arrs] for arrs in scenes]
    tickets = []
    for k, (h, cam) in enumerate(zip(hosts, cams)):
        tickets.append(pipe.submit(h, cam, (0.1, 0.2, 0.3)))
        if k >= 1:  # read the previous frame while this one is in flight
            assert torch.equal(pipe.result(tickets[k - 1]), refs[k - 1])
    assert torch.equal(pipe.result(tickets[-1]), refs[-1])
    assert pipe.instances(tickets[-1])[1] is False or pipe.instances(tickets[-1])[1] == 0
    with pytest.raises(ValueError):
        pipe.result(tickets[0])  # overwritten by frame 2
