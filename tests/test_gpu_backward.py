"""CUDA backward (gs_render_backward, RasterizeGaussians) vs the FP64 oracle.

The bar: per parameter tensor, ||g_gpu - g_ref|| / ||g_ref|| <= 1e-3, with
g_ref the oracle's analytic FP64 gradient (itself pinned to central
differences in test_oracle_grad.py), and directly against FP64 central
differences of the C oracle on sampled parameters.
"""

import numpy as np
import pytest
import torch

import paper_2509_25626_gb300 as gs
from paper_2509_25626_gb300 import SPLAT_DTYPE, SceneTensors
from parity import records_from_oracle
from synth import clustered_scene, orbit_camera, subset_scene
from test_oracle_grad import grad_scene, loss_and_structure

pytestmark = pytest.mark.gpu

DEV = "cuda"
NAMES = ("means", "log_scales", "quats", "opacity_logits", "sh")
BG = (0.1, 0.2, 0.3)


def gpu_grads(sc, cam, dL, bg=BG):
    st = SceneTensors.from_scene(sc, DEV)
    sp = gs.preprocess(st, cam)
    keys, vals, ranges, m, _ = gs.sort(sp, sc.n, cam, max(1024, 64 * sc.n))
    img, T, nc = gs.render(sp, vals, ranges, cam, bg)
    dLt = torch.from_numpy(np.ascontiguousarray(dL, np.float32)).to(DEV)
    grads, dsplat = gs.render_backward(st, cam, sp, vals, ranges, T, nc, dLt, bg)
    torch.cuda.synchronize()
    recs = sp.cpu().numpy().view(SPLAT_DTYPE).reshape(-1)[: sc.n]
    return {k: v.cpu().numpy().astype(np.float64) for k, v in grads.items()}, img.cpu().numpy(), recs


def no_rect_flips(recs, pre):
    ora = records_from_oracle(pre, SPLAT_DTYPE)
    return np.array_equal(recs["rect_lo"], ora["rect_lo"]) and np.array_equal(recs["rect_hi"], ora["rect_hi"])


def rel_err(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30))


def backward_scenes():
    out = [("grad512_s3",) + grad_scene(seed=3), ("grad512_s8",) + grad_scene(seed=8)]
    clu = clustered_scene(20000, seed=6)
    # keep the clustered scene away from the clamps, as the FD scenes are
    clu.opacity_logits[:] = np.clip(clu.opacity_logits, -3.0, 3.0)
    for k in (2, 11):
        out.append((f"clustered20k_orbit{k}", clu, orbit_camera(k, 20, 4.0, 160, 120)))
    return out


@pytest.mark.parametrize("case", [c[0] for c in backward_scenes()])
def test_backward_matches_oracle_gradient(oracle, case):
    from oracle import grad as G
    name, sc, cam = next(c for c in backward_scenes() if c[0] == case)
    dL = np.random.default_rng(1).normal(size=(3, cam.height, cam.width))
    g_gpu, img, recs = gpu_grads(sc, cam, dL)
    pre = oracle.preprocess(sc, cam)
    assert no_rect_flips(recs, pre), "an FP32 rectangle flip changes the lists; pick another seed"
    img_ref, _, g_ref = G.forward_and_grad(sc, cam, dL, BG)
    report = {}
    for k in NAMES:
        e = rel_err(g_gpu[k], g_ref[k])
        report[k] = e
        assert e <= 1e-3, f"{name} {k}: relative error {e:.3e}"
    print(name, {k: f"{v:.2e}" for k, v in report.items()})


def test_backward_matches_central_differences(oracle):
    """Direct check against FP64 central differences of the C oracle."""
    sc, cam = grad_scene(seed=5)
    dL = np.random.default_rng(5).normal(size=(3, cam.height, cam.width))
    g_gpu, _, recs = gpu_grads(sc, cam, dL)
    pre = oracle.preprocess(sc, cam)
    assert no_rect_flips(recs, pre)
    vis = np.nonzero(pre["tiles"] > 0)[0]
    base = loss_and_structure(oracle, sc, cam, dL, BG)[1]
    rng = np.random.default_rng(7)
    for name, arr in zip(NAMES, sc.arrays()):
        fd, gg = [], []
        tried = 0
        while len(fd) < 30 and tried < 300:
            tried += 1
            g = int(rng.choice(vis))
            flat = arr.reshape(arr.shape[0], -1)
            k = int(rng.integers(flat.shape[1]))
            orig = np.float32(flat[g, k])
            h = np.float32(max(1e-5 * abs(float(orig)), 1e-6))
            plus, minus = np.float32(orig + h), np.float32(orig - h)
            flat[g, k] = plus
            lp, sp = loss_and_structure(oracle, sc, cam, dL, BG)
            flat[g, k] = minus
            lm, sm = loss_and_structure(oracle, sc, cam, dL, BG)
            flat[g, k] = orig
            if sp != base or sm != base:
                continue
            fd.append((lp - lm) / (float(plus) - float(minus)))
            gg.append(g_gpu[name].reshape(g_gpu[name].shape[0], -1)[g, k])
        fd, gg = np.array(fd), np.array(gg)
        assert len(fd) >= 15
        e = rel_err(gg, fd)
        assert e <= 1e-3, f"{name}: relative error vs finite differences {e:.3e}"


def test_autograd_function_matches_direct_call():
    sc, cam = grad_scene(seed=3)
    dL = torch.from_numpy(np.random.default_rng(2).normal(size=(3, cam.height, cam.width)).astype(np.float32)).to(DEV)
    params = [torch.from_numpy(np.ascontiguousarray(a)).to(DEV).requires_grad_(True) for a in sc.arrays()]
    img = gs.rasterize(*params, cam, BG, 3)
    (img * dL).sum().backward()
    g_direct, img_direct, _ = gpu_grads(sc, cam, dL.cpu().numpy())
    assert np.array_equal(img.detach().cpu().numpy(), img_direct)
    # the block-level float atomics may add in another order between calls
    for p, k in zip(params, NAMES):
        assert rel_err(p.grad.cpu().numpy().astype(np.float64), g_direct[k]) <= 1e-5


def test_backward_culled_and_empty():
    """Culled Gaussians get zero gradients; an empty scene is fine."""
    sc, cam = grad_scene(seed=3)
    sc.means[:10, 2] = -1.0  # behind the camera
    dL = np.random.default_rng(3).normal(size=(3, cam.height, cam.width))
    g, _, recs = gpu_grads(sc, cam, dL)
    for k in NAMES:
        assert np.all(g[k][:10] == 0)
        assert np.all(np.isfinite(g[k]))
    empty = subset_scene(sc, np.arange(0))
    g0, img0, _ = gpu_grads(empty, cam, dL)
    assert np.allclose(img0[0], BG[0]) and all(v.size == 0 for v in g0.values())


def test_split_backward_equals_combined():
    """gs_render_backward_splats then gs_preprocess_backward give what
    gs_render_backward gives: the per-splat gradients within the reordering
    of float atomics, and the scene gradients from identical per-splat
    gradients bit for bit."""
    sc, cam = clustered_scene(20000, seed=6), orbit_camera(2, 20, 4.0, 160, 120)
    st = SceneTensors.from_scene(sc, DEV)
    sp = gs.preprocess(st, cam)
    _, vals, ranges, _, _ = gs.sort(sp, sc.n, cam, 64 * sc.n)
    _, T, nc = gs.render(sp, vals, ranges, cam, BG)
    dL = torch.randn((3, cam.height, cam.width), generator=torch.Generator().manual_seed(5)).to(DEV)
    grads, dsplat = gs.render_backward(st, cam, sp, vals, ranges, T, nc, dL, BG)
    ds = gs.render_backward_splats(cam, sp, sc.n, vals, ranges, T, nc, dL, BG)
    torch.cuda.synchronize()
    a, b = ds.cpu().numpy().astype(np.float64), dsplat.cpu().numpy().astype(np.float64)
    assert rel_err(a, b) <= 1e-5
    # culled Gaussians (no list) get exact zeros
    tiles = sp[: sc.n].view(torch.int32)[:, 13].cpu().numpy()
    assert np.all(a[tiles == 0] == 0)
    g2 = gs.preprocess_backward(st, cam, sp, dsplat.contiguous())
    for k in NAMES:
        assert torch.equal(g2[k], grads[k]), k
