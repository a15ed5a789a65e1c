"""Seeded scene and camera generators (numpy only).

Every array is float32 and C-contiguous, in the structure-of-arrays layout the
renderer consumes:

    means           [N, 3]      world-space centres
    log_scales      [N, 3]      per-axis log standard deviations
    quats           [N, 4]      rotation quaternions, (w, x, y, z), unit norm
    opacity_logits  [N]         opacity before the sigmoid
    sh              [N, 16, 3]  degree-3 spherical-harmonic coefficients,
                                coefficient-major, RGB-minor

Cameras are pinhole cameras in the OpenCV convention (x right, y down,
z forward).  ``viewmat`` is the 4x4 row-major world-to-camera matrix; pixel
centres sit at integer coordinates, so the optical axis meets the image at
((W - 1) / 2, (H - 1) / 2).

The workload recipes mirror the paper's unbounded-scene workloads (trained
Mip-NeRF 360 and Dr Johnson scenes, Section V-A), which are replaced here by
seeded synthetic scenes of the stated sizes.  Random rotations for cluster
shapes come from a QR factorisation, not from quaternions, so that nothing
here repeats the renderer's own arithmetic.
"""

from __future__ import annotations

import dataclasses
import math

import numpy as np

__all__ = [
    "Camera", "Scene", "CONFIGS", "pinhole_camera", "orbit_camera",
    "uniform_box_scene", "clustered_scene", "slab_scene", "tiny_scene",
    "concat_scenes", "subset_scene",
]


@dataclasses.dataclass
class Camera:
    viewmat: np.ndarray          # (4, 4) float32, row-major, world -> camera
    fx: float
    fy: float
    cx: float
    cy: float
    width: int
    height: int
    tan_fovx: float
    tan_fovy: float

    @property
    def tiles_x(self) -> int:
        return (self.width + 15) // 16

    @property
    def tiles_y(self) -> int:
        return (self.height + 15) // 16

    @property
    def num_tiles(self) -> int:
        return self.tiles_x * self.tiles_y


@dataclasses.dataclass
class Scene:
    means: np.ndarray
    log_scales: np.ndarray
    quats: np.ndarray
    opacity_logits: np.ndarray
    sh: np.ndarray
    sh_degree: int = 3

    @property
    def n(self) -> int:
        return int(self.means.shape[0])

    def arrays(self):
        return (self.means, self.log_scales, self.quats, self.opacity_logits, self.sh)

    def nbytes(self) -> int:
        return sum(a.nbytes for a in self.arrays())


def _f32(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float32))


def pinhole_camera(width: int, height: int, fov_x_deg: float = 60.0,
                   viewmat: np.ndarray | None = None) -> Camera:
    """Square-pixel pinhole camera; the field of view is the horizontal one."""
    tan_fovx = math.tan(math.radians(fov_x_deg) * 0.5)
    fx = width / (2.0 * tan_fovx)
    fy = fx
    tan_fovy = height / (2.0 * fy)
    vm = np.eye(4, dtype=np.float32) if viewmat is None else _f32(viewmat)
    return Camera(vm, float(fx), float(fy), (width - 1) * 0.5, (height - 1) * 0.5,
                  int(width), int(height), float(tan_fovx), float(tan_fovy))


def _look_at(campos: np.ndarray, target: np.ndarray) -> np.ndarray:
    """World-to-camera matrix for a camera at ``campos`` looking at ``target``
    with world +y pointing down in the image (OpenCV axes)."""
    fwd = target - campos
    fwd = fwd / np.linalg.norm(fwd)
    down = np.array([0.0, 1.0, 0.0])
    right = np.cross(down, fwd)
    right = right / np.linalg.norm(right)
    down = np.cross(fwd, right)
    rot = np.stack([right, down, fwd])          # rows: camera axes in world
    vm = np.eye(4)
    vm[:3, :3] = rot
    vm[:3, 3] = -rot @ campos
    return vm.astype(np.float32)


def orbit_camera(k: int, n_poses: int = 20, radius: float = 4.0, width: int = 1600,
                 height: int = 1064, fov_x_deg: float = 60.0, height_y: float = 0.0,
                 arc: float = 2.0 * math.pi) -> Camera:
    """Pose ``k`` of ``n_poses`` on a horizontal circle of ``radius`` around the
    origin, looking at the origin.  Pose 0 sits at (0, height_y, -radius)."""
    phi = arc * k / n_poses
    campos = np.array([radius * math.sin(phi), height_y, -radius * math.cos(phi)])
    return pinhole_camera(width, height, fov_x_deg, _look_at(campos, np.zeros(3)))


def _sh(rng: np.random.Generator, n: int) -> np.ndarray:
    sh = rng.normal(0.0, 0.05, size=(n, 16, 3))
    sh[:, 0, :] = rng.normal(0.0, 0.5, size=(n, 3))
    return _f32(sh)


def _unit_quats(rng: np.random.Generator, n: int) -> np.ndarray:
    q = rng.normal(size=(n, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    return _f32(q)


def uniform_box_scene(n: int = 16384, seed: int = 0) -> Scene:
    """Means x, y ~ U[-1, 1], z ~ U[2, 6]; log-scales N(-4.5, 0.5) per axis;
    unit quaternions from normalised N(0, 1)^4; opacity logits N(0, 1);
    SH DC N(0, 0.5), higher bands N(0, 0.05)."""
    rng = np.random.default_rng(seed)
    means = np.empty((n, 3))
    means[:, 0:2] = rng.uniform(-1.0, 1.0, size=(n, 2))
    means[:, 2] = rng.uniform(2.0, 6.0, size=n)
    log_scales = rng.normal(-4.5, 0.5, size=(n, 3))
    quats = _unit_quats(rng, n)
    logits = rng.normal(0.0, 1.0, size=n)
    return Scene(_f32(means), _f32(log_scales), quats, _f32(logits), _sh(rng, n))


def _random_rotation(rng: np.random.Generator) -> np.ndarray:
    q, r = np.linalg.qr(rng.normal(size=(3, 3)))
    return q * np.sign(np.diag(r))


def clustered_scene(n: int = 3_000_000, seed: int = 1, n_clusters: int = 64,
                    shell_frac: float = 0.2, shell_r: tuple = (10.0, 50.0),
                    ball_r: float = 3.0, axis_std: tuple = (0.05, 0.8),
                    log_scale_centre: float = -5.0, log_scale_t_scale: float = 0.25,
                    log_scale_clip: tuple = (-12.0, -2.0), opacity_std: float = 1.5,
                    opacity_centre: float = 0.0) -> Scene:
    """Mixture of ``n_clusters`` anisotropic Gaussian clusters (centres uniform
    in a ball of radius ``ball_r``, random orientation, axis standard
    deviations log-uniform in ``axis_std``) plus a ``shell_frac`` share of
    points uniform in direction at radius U[shell_r].  Log-scales are
    ``log_scale_centre`` + ``log_scale_t_scale`` * Student-t(3) per axis,
    clipped to ``log_scale_clip``; opacity logits N(``opacity_centre``,
    ``opacity_std``); SH as in ``uniform_box_scene``.

    With the defaults, at 3M points and 1600x1064 on the orbit poses, each
    16x16 tile overlaps about 1.4e3 Gaussians on average with variance/mean^2
    of 0.5-0.7, the density the paper reports for its unbounded scenes
    (Table III: mean 1189, variance 614608)."""
    rng = np.random.default_rng(seed)
    n_shell = int(round(n * shell_frac))
    n_clu = n - n_shell
    # cluster centres uniform in a ball
    d = rng.normal(size=(n_clusters, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    centres = d * (ball_r * rng.uniform(0, 1, size=(n_clusters, 1)) ** (1.0 / 3.0))
    rots = np.stack([_random_rotation(rng) for _ in range(n_clusters)])
    stds = np.exp(rng.uniform(np.log(axis_std[0]), np.log(axis_std[1]), size=(n_clusters, 3)))
    label = rng.integers(0, n_clusters, size=n_clu)
    local = rng.normal(size=(n_clu, 3)) * stds[label]
    pts = centres[label] + np.einsum("nij,nj->ni", rots[label], local)
    # background shell
    d = rng.normal(size=(n_shell, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    shell = d * rng.uniform(shell_r[0], shell_r[1], size=(n_shell, 1))
    means = np.concatenate([pts, shell], axis=0)
    perm = rng.permutation(n)
    means = means[perm]
    log_scales = np.clip(log_scale_centre + log_scale_t_scale * rng.standard_t(3, size=(n, 3)),
                         *log_scale_clip)
    quats = _unit_quats(rng, n)
    logits = rng.normal(opacity_centre, opacity_std, size=n)
    return Scene(_f32(means), _f32(log_scales), quats, _f32(logits), _sh(rng, n))


def slab_scene(n: int = 6_000_000, seed: int = 5, slab_frac: float = 0.5) -> Scene:
    """Load-imbalance stress scene: ``slab_frac`` of the points packed into a
    dense occluding slab x, y in [-0.15, 0.15], z in [2.0, 2.2] with the
    clustered scene's scale and opacity laws; the rest as ``clustered_scene``."""
    n_slab = int(round(n * slab_frac))
    base = clustered_scene(n - n_slab, seed=seed)
    rng = np.random.default_rng(seed + 1000)
    means = np.empty((n_slab, 3))
    means[:, 0:2] = rng.uniform(-0.15, 0.15, size=(n_slab, 2))
    means[:, 2] = rng.uniform(2.0, 2.2, size=n_slab)
    log_scales = np.clip(-5.0 + 0.25 * rng.standard_t(3, size=(n_slab, 3)), -12.0, -2.0)
    slab = Scene(_f32(means), _f32(log_scales), _unit_quats(rng, n_slab),
                 _f32(rng.normal(0.0, 1.5, size=n_slab)), _sh(rng, n_slab))
    return concat_scenes([base, slab])


def tiny_scene(n: int, seed: int, width: int, height: int, fov_x_deg: float = 60.0,
               z_range: tuple = (1.0, 5.0), log_scale: tuple = (-3.5, 0.6),
               spill: float = 1.2, near_frac: float = 0.0,
               opacity_std: float = 1.0) -> tuple[Scene, Camera]:
    """Small scene in front of a camera at the origin, for exact tests.

    Means fill the view frustum (``spill`` > 1 puts some just outside it);
    ``near_frac`` of them are moved to z in [-0.5, 0.3] to exercise the
    near-plane cull."""
    rng = np.random.default_rng(seed)
    cam = pinhole_camera(width, height, fov_x_deg)
    z = rng.uniform(z_range[0], z_range[1], size=n)
    n_near = int(round(n * near_frac))
    if n_near:
        z[:n_near] = rng.uniform(-0.5, 0.3, size=n_near)
    x = rng.uniform(-spill, spill, size=n) * cam.tan_fovx * np.abs(z)
    y = rng.uniform(-spill, spill, size=n) * cam.tan_fovy * np.abs(z)
    means = np.stack([x, y, z], axis=1)
    log_scales = rng.normal(log_scale[0], log_scale[1], size=(n, 3))
    quats = _unit_quats(rng, n)
    logits = rng.normal(0.0, opacity_std, size=n)
    return Scene(_f32(means), _f32(log_scales), quats, _f32(logits), _sh(rng, n)), cam


def needle_scene(n: int, seed: int, width: int, height: int) -> tuple[Scene, Camera]:
    """Needle-like Gaussians at every orientation in front of a camera at the
    origin: one long axis (log-scale N(-1.8, 0.3)) and two thin ones
    (N(-6, 0.3)), uniformly random rotations, so that their projected
    ellipses are thin and slanted at every angle."""
    rng = np.random.default_rng(seed)
    cam = pinhole_camera(width, height, 60.0)
    z = rng.uniform(1.5, 4.0, size=n)
    x = rng.uniform(-1.1, 1.1, size=n) * cam.tan_fovx * z
    y = rng.uniform(-1.1, 1.1, size=n) * cam.tan_fovy * z
    means = np.stack([x, y, z], axis=1)
    log_scales = np.stack([rng.normal(-1.8, 0.3, size=n), rng.normal(-6.0, 0.3, size=n),
                           rng.normal(-6.0, 0.3, size=n)], axis=1)
    quats = _unit_quats(rng, n)
    logits = rng.normal(1.0, 1.0, size=n)
    return Scene(_f32(means), _f32(log_scales), quats, _f32(logits), _sh(rng, n)), cam


def concat_scenes(scenes) -> Scene:
    return Scene(*[_f32(np.concatenate(parts, axis=0)) for parts in zip(*[s.arrays() for s in scenes])])


def subset_scene(scene: Scene, idx) -> Scene:
    return Scene(*[_f32(a[idx]) for a in scene.arrays()], sh_degree=scene.sh_degree)


# Named workloads.  Sizes follow the benchmark configurations; every call is
# seeded so the oracle and the CUDA path see identical arrays.
CONFIGS = {
    "fwd_16k_256": dict(scene=lambda: uniform_box_scene(16384, seed=0),
                        cameras=lambda: [pinhole_camera(256, 256, 60.0)]),
    "fwd_3m_1600x1064": dict(scene=lambda: clustered_scene(3_000_000, seed=1),
                             cameras=lambda: [orbit_camera(k, 20, 4.0, 1600, 1064) for k in range(20)]),
    "bwd_1m_1237x822": dict(scene=lambda: clustered_scene(1_000_000, seed=3),
                            cameras=lambda: [orbit_camera(k, 20, 4.0, 1237, 822) for k in range(20)]),
    "slab_6m_3840x2160x8": dict(scene=lambda: slab_scene(6_000_000, seed=5),
                                cameras=lambda: [orbit_camera(k, 8, 4.0, 3840, 2160,
                                                              arc=math.radians(40.0)) for k in range(8)]),
}
