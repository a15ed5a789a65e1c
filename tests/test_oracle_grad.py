"""Pins for the FP64 gradient oracle (``oracle/grad.py``).

1. Its differentiable forward reproduces the C oracle's image and final
   transmittance (to rounding), so it differentiates the same function.
2. Its gradients equal FP64 central finite differences of the C oracle's
   loss sum(dL/dpixel * image) for randomly chosen scalar parameters of every
   tensor (means, log scales, quaternions, opacity logits, SH).  A sample
   whose +/- perturbation changes any discrete decision (a rectangle, a skip,
   a stop) is discarded: the function is piecewise smooth and the finite
   difference straddles a jump there.
No GPU needed.
"""

import numpy as np
import pytest

from synth import Scene, tiny_scene

pytestmark = pytest.mark.filterwarnings("ignore::RuntimeWarning")


def grad_scene(n=512, seed=3, w=64, h=64):
    """A 512-Gaussian 64x64 sub-scene away from the clamps: opacity logits in
    [-3, 3] (alpha stays below the 0.99 clamp), colour well above 0."""
    sc, cam = tiny_scene(n, seed, w, h, log_scale=(-3.0, 0.5))
    rng = np.random.default_rng(seed + 100)
    sc.opacity_logits[:] = np.clip(sc.opacity_logits, -3.0, 3.0)
    sc.sh[:, 0, :] = np.abs(rng.normal(0.0, 0.5, size=(n, 3))).astype(np.float32) + 0.3
    return sc, cam


def loss_and_structure(oracle, sc, cam, dL, bg):
    pre, srt, img = oracle.frame(sc, cam, bg=bg)
    loss = float((img["color"] * dL).sum())
    struct = (pre["rect"].tobytes(), img["n_contrib"].tobytes(), img["n_eval"].tobytes())
    return loss, struct


def test_grad_forward_matches_c_oracle(oracle):
    from oracle import grad as G
    sc, cam = grad_scene()
    bg = (0.1, 0.2, 0.3)
    dL = np.random.default_rng(0).normal(size=(3, cam.height, cam.width))
    img, T, _ = G.forward_and_grad(sc, cam, dL, bg)
    _, _, ora = oracle.frame(sc, cam, bg=bg)
    np.testing.assert_allclose(img, ora["color"], atol=1e-12)
    np.testing.assert_allclose(T, ora["final_T"], atol=1e-12)


@pytest.mark.parametrize("seed", [3, 8])
def test_grad_matches_central_differences(oracle, seed):
    from oracle import grad as G
    sc, cam = grad_scene(seed=seed)
    bg = (0.1, 0.2, 0.3)
    rng = np.random.default_rng(seed)
    dL = rng.normal(size=(3, cam.height, cam.width))
    _, _, ag = G.forward_and_grad(sc, cam, dL, bg)
    pre = oracle.preprocess(sc, cam)
    vis = np.nonzero(pre["tiles"] > 0)[0]
    base_struct = loss_and_structure(oracle, sc, cam, dL, bg)[1]
    names = ("means", "log_scales", "quats", "opacity_logits", "sh")
    for name, arr in zip(names, sc.arrays()):
        fd_vals, ag_vals = [], []
        tried = 0
        while len(fd_vals) < 40 and tried < 400:
            tried += 1
            g = int(rng.choice(vis))
            flat = arr.reshape(arr.shape[0], -1)
            k = int(rng.integers(flat.shape[1]))
            if name == "sh" and k // 3 >= (sc.sh_degree + 1) ** 2:
                continue
            orig = np.float32(flat[g, k])
            h = np.float32(max(1e-5 * abs(float(orig)), 1e-6))
            plus, minus = np.float32(orig + h), np.float32(orig - h)
            flat[g, k] = plus
            lp, sp = loss_and_structure(oracle, sc, cam, dL, bg)
            flat[g, k] = minus
            lm, sm = loss_and_structure(oracle, sc, cam, dL, bg)
            flat[g, k] = orig
            if sp != base_struct or sm != base_struct:
                continue  # a discrete decision flipped inside the stencil
            fd_vals.append((lp - lm) / (float(plus) - float(minus)))
            ag_vals.append(ag[name].reshape(ag[name].shape[0], -1)[g, k])
        fd_vals, ag_vals = np.array(fd_vals), np.array(ag_vals)
        assert len(fd_vals) >= 20, f"{name}: too few clean samples"
        scale = np.sqrt(np.mean(ag_vals ** 2)) + 1e-12
        err = np.abs(fd_vals - ag_vals)
        assert np.all(err <= 1e-4 * np.abs(ag_vals) + 1e-5 * scale), \
            f"{name}: max err {err.max():.3e} (scale {scale:.3e})"
