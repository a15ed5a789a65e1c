"""FP64 analytic gradient of the forward pass, for checking the CUDA backward.

TEST INFRASTRUCTURE ONLY (tests and the smoke check import it; the CUDA
library never does).

The forward is rewritten in plain PyTorch CPU ops in float64 -- the same
definitions as ``gs_oracle.c`` (Section II-B preprocessing with the EWA
projection and degree-3 SH colour; Eq. 1 blending with the kernel's alpha,
the 1/255 skip, the 0.99 clamp and the 1e-4 stop of Algorithm 1 / Appendix
B) -- and autograd supplies the chain rule.  The discrete structure (tile
rectangles, the sorted per-tile lists, which splats are skipped, where each
pixel stops) is taken from the C oracle and held fixed, as the derivative of
a piecewise-smooth function is that of the piece it is on.  The forward here
is pinned to the C oracle's image, and the gradient to central differences
of the C oracle, by ``tests/test_oracle_grad.py``.
"""

from __future__ import annotations

import math

import numpy as np
import torch

from . import oracle as O

F64 = torch.float64
ALPHA_MAX = 0.99
ALPHA_MIN = 1.0 / 255.0
T_MIN = 1e-4


def sh_basis(d: torch.Tensor) -> torch.Tensor:
    """[N, 16] real SH (Condon-Shortley phase) of unit directions d [N, 3],
    in their textbook Cartesian forms."""
    x, y, z = d[:, 0], d[:, 1], d[:, 2]
    pi = math.pi
    a1 = math.sqrt(3 / (4 * pi))
    cols = [
        torch.full_like(x, 1 / (2 * math.sqrt(pi))),
        -a1 * y, a1 * z, -a1 * x,
        0.5 * math.sqrt(15 / pi) * x * y,
        -0.5 * math.sqrt(15 / pi) * y * z,
        0.25 * math.sqrt(5 / pi) * (3 * z * z - 1),
        -0.5 * math.sqrt(15 / pi) * x * z,
        0.25 * math.sqrt(15 / pi) * (x * x - y * y),
        -0.25 * math.sqrt(35 / (2 * pi)) * y * (3 * x * x - y * y),
        0.5 * math.sqrt(105 / pi) * x * y * z,
        -0.25 * math.sqrt(21 / (2 * pi)) * y * (5 * z * z - 1),
        0.25 * math.sqrt(7 / pi) * z * (5 * z * z - 3),
        -0.25 * math.sqrt(21 / (2 * pi)) * x * (5 * z * z - 1),
        0.25 * math.sqrt(105 / pi) * z * (x * x - y * y),
        -0.25 * math.sqrt(35 / (2 * pi)) * x * (x * x - 3 * y * y),
    ]
    return torch.stack(cols, dim=1)


def preprocess(means, log_scales, quats, logits, sh, cam, sh_degree: int = 3):
    """Differentiable projection of every Gaussian (culling is decided by the
    C oracle and applied by the caller): xy [N,2], conic [N,3], opacity [N],
    rgb [N,3]."""
    rec = O.camera_record(cam).astype(np.float64)
    V = torch.tensor(rec[:16].reshape(4, 4), dtype=F64)
    fx, fy, cx, cy = (float(v) for v in rec[16:20])
    tanx, tany = float(rec[22]), float(rec[23])
    W = V[:3, :3]
    t = means @ W.T + V[:3, 3]
    tx, ty, tz = t[:, 0], t[:, 1], t[:, 2]
    q = quats / torch.linalg.norm(quats, dim=1, keepdim=True)
    w, x, y, z = q[:, 0], q[:, 1], q[:, 2], q[:, 3]
    R = torch.stack([
        torch.stack([1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)], 1),
        torch.stack([2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)], 1),
        torch.stack([2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)], 1),
    ], 1)
    S2 = torch.diag_embed(torch.exp(2 * log_scales))
    Sigma = R @ S2 @ R.transpose(1, 2)
    limx, limy = 1.3 * tanx, 1.3 * tany
    txc = torch.clamp(tx / tz, -limx, limx) * tz
    tyc = torch.clamp(ty / tz, -limy, limy) * tz
    zero = torch.zeros_like(tz)
    J = torch.stack([
        torch.stack([fx / tz, zero, -fx * txc / (tz * tz)], 1),
        torch.stack([zero, fy / tz, -fy * tyc / (tz * tz)], 1),
    ], 1)
    T = J @ W
    C2 = T @ Sigma @ T.transpose(1, 2)
    s00 = C2[:, 0, 0] + 0.3
    s01 = C2[:, 0, 1]
    s11 = C2[:, 1, 1] + 0.3
    det = s00 * s11 - s01 * s01
    conic = torch.stack([s11 / det, -s01 / det, s00 / det], 1)
    xy = torch.stack([fx * tx / tz + cx, fy * ty / tz + cy], 1)
    campos = -(W.T @ V[:3, 3])
    dvec = means - campos
    d = dvec / torch.linalg.norm(dvec, dim=1, keepdim=True)
    Y = sh_basis(d)
    ncoef = (sh_degree + 1) ** 2
    raw = torch.einsum("nk,nkc->nc", Y[:, :ncoef], sh[:, :ncoef, :]) + 0.5
    rgb = torch.clamp(raw, min=0.0)
    opacity = torch.sigmoid(logits)
    return xy, conic, opacity, rgb


def render(xy, conic, opacity, rgb, srt: dict, cam, bg):
    """Differentiable tiled compositing on the fixed per-tile lists; the
    skip and stop decisions are made on detached values."""
    Wd, Hd = int(cam.width), int(cam.height)
    tiles_x = (Wd + 15) // 16
    out = torch.zeros((3, Hd, Wd), dtype=F64)
    out_T = torch.ones((Hd, Wd), dtype=F64)
    bgt = torch.tensor(bg, dtype=F64)
    ranges = srt["ranges"]
    vals = srt["vals"].astype(np.int64)
    pieces = []
    for tile in range(ranges.shape[0]):
        s, e = int(ranges[tile, 0]), int(ranges[tile, 1])
        ty, tx = divmod(tile, tiles_x)
        ys = torch.arange(ty * 16, min(ty * 16 + 16, Hd), dtype=F64)
        xs = torch.arange(tx * 16, min(tx * 16 + 16, Wd), dtype=F64)
        if len(ys) == 0 or len(xs) == 0:
            continue
        py, px = torch.meshgrid(ys, xs, indexing="ij")
        px, py = px.reshape(-1), py.reshape(-1)
        if e <= s:
            pieces.append((ty, tx, len(ys), len(xs), bgt[:, None].expand(3, len(px)), torch.ones(len(px), dtype=F64)))
            continue
        ids = torch.from_numpy(vals[s:e])
        dx = xy[ids, 0][None, :] - px[:, None]
        dy = xy[ids, 1][None, :] - py[:, None]
        a, b, c = conic[ids, 0][None], conic[ids, 1][None], conic[ids, 2][None]
        power = -0.5 * (a * dx * dx + c * dy * dy) - b * dx * dy
        alpha = torch.clamp(opacity[ids][None] * torch.exp(power), max=ALPHA_MAX)
        with torch.no_grad():
            keep = (power <= 0) & (alpha >= ALPHA_MIN)
            one_minus = torch.where(keep, 1 - alpha, torch.ones_like(alpha))
            T_excl = torch.cumprod(torch.cat([torch.ones_like(one_minus[:, :1]), one_minus[:, :-1]], 1), 1)
            stop = keep & (T_excl * (1 - alpha) < T_MIN)
            L = stop.shape[1]
            idx = torch.arange(L)[None].expand_as(stop)
            first = torch.where(stop, idx, torch.full_like(idx, L)).min(dim=1).values
            blend = keep & (idx < first[:, None])
        a_eff = torch.where(blend, alpha, torch.zeros_like(alpha))
        om = 1 - a_eff
        T_ex = torch.cumprod(torch.cat([torch.ones_like(om[:, :1]), om[:, :-1]], 1), 1)
        wgt = a_eff * T_ex
        col = wgt @ rgb[ids]                      # [P, 3]
        T_fin = T_ex[:, -1] * om[:, -1]
        col = col + T_fin[:, None] * bgt[None]
        pieces.append((ty, tx, len(ys), len(xs), col.T, T_fin))
    rows = []
    for ty in range((Hd + 15) // 16):
        rows.append([p for p in pieces if p[0] == ty])
    img_rows, T_rows = [], []
    for row in rows:
        row = sorted(row, key=lambda p: p[1])
        img_rows.append(torch.cat([p[4].reshape(3, p[2], p[3]) for p in row], 2))
        T_rows.append(torch.cat([p[5].reshape(p[2], p[3]) for p in row], 1))
    out = torch.cat(img_rows, 1)
    out_T = torch.cat(T_rows, 0)
    return out, out_T


def clip_to_tile_rows(pre: dict, ty0: int, ty1: int) -> dict:
    """The preprocess output with every rectangle clipped to tile rows
    [ty0, ty1): the tiles of those rows keep exactly their lists and order
    (a list holds the Gaussians whose rectangle covers the tile, sorted by
    depth then id), and no other tile has any."""
    clip = dict(pre)
    rect = pre["rect"].copy()
    rect[:, 1] = np.maximum(rect[:, 1], ty0)
    rect[:, 3] = np.minimum(rect[:, 3], ty1)
    keep = (pre["tiles"] > 0) & (rect[:, 3] > rect[:, 1])
    clip["rect"] = np.where(keep[:, None], rect, 0).astype(np.int32)
    clip["tiles"] = np.where(keep, (rect[:, 2] - rect[:, 0]) * (rect[:, 3] - rect[:, 1]), 0).astype(np.int32)
    return clip


def forward_and_grad(scene, cam, dL_dcolor: np.ndarray, bg=(0.0, 0.0, 0.0), tile_rows: tuple | None = None):
    """Image and d(sum dL_dcolor * image)/d(scene parameters), all FP64.
    Returns (image [3,H,W], final T [H,W], grads dict with means, log_scales,
    quats, opacity_logits, sh).  With tile_rows = (ty0, ty1) only those tile
    rows are rendered (pixel rows [16 ty0, 16 ty1); elsewhere the image is
    the background) and differentiated, for a dL_dcolor that is zero outside
    them: the same gradient at a fraction of the cost."""
    pre = O.preprocess(scene, cam)
    if tile_rows is not None:
        pre = clip_to_tile_rows(pre, *tile_rows)
    srt = O.duplicate_sort(pre, cam)
    params = {k: torch.tensor(np.asarray(a, np.float64), dtype=F64, requires_grad=True)
              for k, a in zip(("means", "log_scales", "quats", "opacity_logits", "sh"), scene.arrays())}
    # only visible Gaussians are differentiated (culled ones appear in no list
    # and may sit on the camera plane, where the projection is singular)
    n = scene.n
    vi = torch.from_numpy(np.nonzero(pre["tiles"] > 0)[0])
    sub = [params[k].index_select(0, vi) for k in ("means", "log_scales", "quats", "opacity_logits", "sh")]
    xy_v, conic_v, op_v, rgb_v = preprocess(*sub, cam, scene.sh_degree)
    xy = torch.zeros((n, 2), dtype=F64).index_copy(0, vi, xy_v)
    conic = torch.zeros((n, 3), dtype=F64).index_copy(0, vi, conic_v)
    op = torch.zeros(n, dtype=F64).index_copy(0, vi, op_v)
    rgb = torch.zeros((n, 3), dtype=F64).index_copy(0, vi, rgb_v)
    img, T = render(xy, conic, op, rgb, srt, cam, bg)
    loss = (img * torch.from_numpy(np.asarray(dL_dcolor, np.float64))).sum()
    loss.backward()
    grads = {k: v.grad.numpy().copy() for k, v in params.items()}
    return img.detach().numpy(), T.detach().numpy(), grads
