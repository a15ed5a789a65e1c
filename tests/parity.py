"""Comparison helpers for the GPU parity tests (CUDA path vs FP64 oracle).

Tolerances (written here, used by every parity test):

IMAGE_ATOL = 2e-4
    Absolute per-channel pixel tolerance in FP32 (the stated bar).
TAU_ALPHA, TAU_T
    Log-space margins under which an alpha-threshold or transmittance-stop
    decision counts as "near": the FP32 path may take it the other way.
    A pixel is excluded from the 2e-4 check only if taking such a near
    decision the other way moves it by more than IMAGE_ATOL / 2 (the oracle's
    flip_impact: the pixel walked again with that one decision flipped, every
    later decision re-evaluated, so a flip that moves a later stop counts in
    full), and excluded from the exact n_contrib check if it has any near
    decision.
    The FP32 error of the exponent from its own arithmetic is about 1e-6
    (ex2.approx relative error 2^-22, conic rounding); TAU_ALPHA = 1e-4
    leaves a factor of ~100.  Transmittance accumulates one rounding per
    blend (<= ~2000 blends before T < 1e-4), so TAU_T = 1e-3.  On top, a
    splat's FP32 pixel coordinates carry a rounding that grows with |x|; the
    oracle widens each margin by |d power / d x| POS_EPS (|x| + 1), with
    POS_EPS = 2^-23 (two ulps) when the GPU renders the oracle's own
    coordinates rounded to FP32 and 2^-21 when it projects them itself.
EDGE_TOL_PX, RADIUS_TOL
    Integer decisions of the preprocess (radius, tile rectangle) may flip
    only for Gaussians whose FP64 value lies this close to the boundary.
"""

from __future__ import annotations

import math

import numpy as np

IMAGE_ATOL = 2e-4
TAU_ALPHA = 1e-4
TAU_T = 1e-3
POS_EPS_RENDER = 2.0 ** -23
POS_EPS_E2E = 2.0 ** -21
RADIUS_TOL = 1e-4      # |3 sqrt(lambda) - k| below this (relative to value) may flip
EDGE_TOL_PX = 2e-3     # rectangle edges within this many pixels of a tile boundary may flip
XY_TOL_REL = 2e-6      # |x_gpu - x| <= XY_TOL_REL * (|x| + fx) pixels

LOG2E = math.log2(math.e)
KW = math.sqrt(LOG2E / 2.0)


def records_from_oracle(pre: dict, splat_dtype) -> np.ndarray:
    """The oracle's preprocess output in the CUDA library's 64-byte record
    layout (float32), so that gs_sort / gs_render can run on oracle inputs."""
    n = pre["xy"].shape[0]
    rec = np.zeros(n, splat_dtype)
    vis = pre["tiles"] > 0
    s00, s01, s11 = (pre["cov2d"][:, k] for k in range(3))
    with np.errstate(divide="ignore", invalid="ignore"):
        det = s00 * s11 - s01 * s01
        w00 = KW * np.sqrt(s11 / det)
        w01 = -w00 * s01 / s11
        w11 = KW / np.sqrt(s11)
        lg2o = np.log2(pre["opacity"])
    rec["x"] = np.where(vis, pre["xy"][:, 0], 0)
    rec["y"] = np.where(vis, pre["xy"][:, 1], 0)
    rec["w00"] = np.where(vis, w00, 0)
    rec["w01"] = np.where(vis, w01, 0)
    rec["w11"] = np.where(vis, w11, 0)
    rec["log2_opacity"] = np.where(vis, lg2o, 0)
    for k, ch in enumerate("rgb"):
        rec[ch] = np.where(vis, pre["rgb"][:, k], 0)
    rec["depth"] = pre["depth32"]
    rec["radius"] = np.where(vis, pre["radius"], 0)
    rec["tiles_touched"] = pre["tiles"].astype(np.uint32)
    r = pre["rect"].astype(np.uint32)
    rec["rect_lo"] = np.where(vis, r[:, 0] | (r[:, 1] << 16), 0)
    rec["rect_hi"] = np.where(vis, r[:, 2] | (r[:, 3] << 16), 0)
    hx, hy = cull_box(pre)
    rec["cull_hx"] = np.where(vis, hx * (1 + 2.0 ** -10) + 1.0 / 64, -1.0)
    rec["cull_hy"] = np.where(vis, hy * (1 + 2.0 ** -10) + 1.0 / 64, -1.0)
    rec["cull_hx"][vis & (hx < 0)] = -1.0
    rec["cull_hy"][vis & (hy < 0)] = -1.0
    return rec


def cull_box(pre: dict):
    """Half-extents of the bounding box of the region where alpha = o
    exp(-d^T Sigma'^-1 d / 2) reaches 1/255: sqrt(2 ln(255 o) Sigma'_xx) and
    sqrt(2 ln(255 o) Sigma'_yy); -1 where 255 o <= 1 (nowhere)."""
    with np.errstate(divide="ignore", invalid="ignore"):
        r2 = 2.0 * np.log(255.0 * pre["opacity"])
        hx = np.where(r2 > 0, np.sqrt(np.maximum(r2, 0) * pre["cov2d"][:, 0]), -1.0)
        hy = np.where(r2 > 0, np.sqrt(np.maximum(r2, 0) * pre["cov2d"][:, 2]), -1.0)
    return hx, hy


def conic_from_record(rec: np.ndarray) -> np.ndarray:
    """Sigma'^-1 entries (a, b, c) implied by a record's factor."""
    w00, w01, w11 = (rec[k].astype(np.float64) for k in ("w00", "w01", "w11"))
    s = 1.0 / (KW * KW)
    return np.stack([w00 * w00 * s, w00 * w01 * s, (w01 * w01 + w11 * w11) * s], axis=1)


def rect_of(rec: np.ndarray) -> np.ndarray:
    lo, hi = rec["rect_lo"].astype(np.int64), rec["rect_hi"].astype(np.int64)
    return np.stack([lo & 0xFFFF, lo >> 16, hi & 0xFFFF, hi >> 16], axis=1)


def ambiguous_gaussians(pre: dict, cam) -> np.ndarray:
    """Gaussians whose radius or rectangle may legitimately differ in FP32."""
    rr = 3.0 * np.sqrt(np.maximum(pre["radius"].astype(np.float64), 1.0))  # scale of the radius value
    near_r = pre["rad_dist"] < RADIUS_TOL * np.maximum(rr * rr / 9.0, 1.0)
    scale = np.abs(pre["xy"]).max(axis=1) + float(cam.fx)
    near_e = pre["edge_dist"] < np.maximum(EDGE_TOL_PX, XY_TOL_REL * scale * 4)
    return near_r | near_e


def compare_preprocess(gpu: np.ndarray, pre: dict, cam) -> dict:
    """Element-wise comparison of GPU records with the oracle.  Returns a
    report; raises AssertionError on a mismatch outside the stated bounds."""
    amb = ambiguous_gaussians(pre, cam)
    depth_bits_gpu = gpu["depth"].view(np.uint32)
    depth_bits_ora = pre["depth32"].view(np.uint32)
    assert np.array_equal(depth_bits_gpu, depth_bits_ora), "FP32 depth (sort key) differs"
    vis_o = pre["tiles"] > 0
    vis_g = gpu["tiles_touched"] > 0
    flip = (vis_o != vis_g)
    assert not np.any(flip & ~amb), f"visibility differs on {np.sum(flip & ~amb)} non-ambiguous Gaussians"
    both = vis_o & vis_g
    rect_g = rect_of(gpu)
    bad_int = both & ((gpu["radius"] != pre["radius"]) | np.any(rect_g != pre["rect"], axis=1) |
                      (gpu["tiles_touched"].astype(np.int64) != pre["tiles"]))
    assert not np.any(bad_int & ~amb), f"radius/rect differ on {np.sum(bad_int & ~amb)} non-ambiguous Gaussians"
    b = both
    xy_err = np.abs(np.stack([gpu["x"], gpu["y"]], 1).astype(np.float64) - pre["xy"])[b]
    xy_scale = (np.abs(pre["xy"][b]).max(axis=1) + float(cam.fx))[:, None]
    assert np.all(xy_err <= XY_TOL_REL * xy_scale + 1e-6), f"xy error {xy_err.max():.3e}"
    conic_g = conic_from_record(gpu)[b]
    conic_o = pre["conic"][b]
    cnorm = np.abs(conic_o).max(axis=1, keepdims=True)
    conic_rel = np.abs(conic_g - conic_o) / cnorm
    assert np.all(conic_rel <= 1e-4), f"conic relative error {conic_rel.max():.3e}"
    rgb_err = np.abs(np.stack([gpu["r"], gpu["g"], gpu["b"]], 1) - pre["rgb"])[b]
    assert np.all(rgb_err <= 2e-5), f"rgb error {rgb_err.max():.3e}"
    op_err = np.abs(np.exp2(gpu["log2_opacity"].astype(np.float64)) - pre["opacity"])[b]
    assert np.all(op_err <= 1e-6), f"opacity error {op_err.max():.3e}"
    # the culling box must contain the exact alpha >= 1/255 region, and be tight
    hx, hy = cull_box(pre)
    with np.errstate(divide="ignore"):
        rho_margin = np.abs(np.log(255.0 * pre["opacity"]))
    firm = b & (rho_margin > 1e-5)
    for got, want in ((gpu["cull_hx"], hx), (gpu["cull_hy"], hy)):
        g, w = got[firm].astype(np.float64), want[firm]
        assert np.all((w < 0) == (g < 0)), "culling box emptiness differs"
        pos = w >= 0
        assert np.all(g[pos] >= w[pos] * (1 - 1e-6)), "culling box smaller than the alpha >= 1/255 region"
        assert np.all(g[pos] <= w[pos] * 1.002 + 0.02), "culling box looser than its stated slack"
    lg_err = np.abs(gpu["log2_opacity"][b].astype(np.float64) - np.log2(pre["opacity"][b]))
    assert np.all(lg_err <= 1e-5 * np.maximum(1.0, np.abs(np.log2(pre["opacity"][b])))), \
        f"log2 opacity error {lg_err.max():.3e}"
    return dict(n=len(pre["tiles"]), visible=int(vis_o.sum()), ambiguous=int(amb.sum()),
                int_flips=int(np.sum(bad_int) + np.sum(flip)), xy_err=float(xy_err.max(initial=0)),
                conic_rel=float(conic_rel.max(initial=0)), rgb_err=float(rgb_err.max(initial=0)))


def compare_images(img: np.ndarray, final_T: np.ndarray, n_contrib: np.ndarray, ora: dict,
                   exclude: np.ndarray | None = None, max_excluded_frac: float = 0.01) -> dict:
    """GPU image vs oracle: 2e-4 absolute on every pixel except those where a
    near-threshold decision could move the value by more than half the
    tolerance; n_contrib exact where no decision was near."""
    near_amb = ora["flip_impact"] > IMAGE_ATOL / 2
    amb = near_amb if exclude is None else (near_amb | exclude)
    err = np.abs(img.astype(np.float64) - ora["color"]).max(axis=0)
    bad = (err > IMAGE_ATOL) & ~amb
    assert not np.any(bad), (f"{bad.sum()} pixels exceed {IMAGE_ATOL}: max {err[bad].max():.3e} "
                             f"at {np.argwhere(bad)[:5].tolist()}")
    t_err = np.abs(final_T.astype(np.float64) - ora["final_T"])
    assert np.all((t_err <= IMAGE_ATOL) | amb), f"final_T error {t_err[~amb].max():.3e}"
    exact = ora["near"] == 0
    if exclude is not None:
        exact &= ~exclude
    nc_bad = (n_contrib.astype(np.int64) != ora["n_contrib"]) & exact
    assert not np.any(nc_bad), f"n_contrib differs on {nc_bad.sum()} pixels with no near decision"
    frac = float(near_amb.mean())
    assert frac <= max_excluded_frac, f"{frac:.4f} of pixels excluded as ambiguous"
    return dict(max_err=float(err[~amb].max(initial=0)), excluded=int(near_amb.sum()),
                excluded_flip_tiles=int(0 if exclude is None else exclude.sum()), near=int((~exact).sum()),
                pixels=int(err.size), n_contrib_mismatch=int(((n_contrib != ora["n_contrib"]) & ~exact).sum()))


def flip_tile_mask(recs: np.ndarray, pre: dict, flipped: np.ndarray, cam, rows=(0, None)) -> np.ndarray:
    """Pixels of the tiles in the symmetric difference of the GPU's and the
    oracle's rectangle for each Gaussian whose rectangle flipped (each such
    Gaussian must be flagged ambiguous; those tiles' lists legitimately
    differ by that one Gaussian)."""
    r0 = rows[0]
    r1 = cam.height if rows[1] is None else rows[1]
    mask = np.zeros((r1 - r0, cam.width), bool)
    rg = rect_of(recs)
    for g in flipped:
        a = set((tx, ty) for ty in range(rg[g, 1], rg[g, 3]) for tx in range(rg[g, 0], rg[g, 2]))
        x0, y0, x1, y1 = pre["rect"][g]
        b = set((tx, ty) for ty in range(y0, y1) for tx in range(x0, x1))
        for tx, ty in a ^ b:
            ya, yb = max(ty * 16, r0), min(ty * 16 + 16, r1)
            if ya < yb:
                mask[ya - r0:yb - r0, tx * 16:tx * 16 + 16] = True
    return mask


def check_sorted_output(keys: np.ndarray, vals: np.ndarray, ranges: np.ndarray, m: int, recs: np.ndarray,
                        tiles_x: int):
    """Properties of a sort that hold at any size (used where the oracle's
    full sort would be too slow): keys ascending, each instance's tile inside
    its Gaussian's rectangle with its depth bits, ranges consistent,
    per-Gaussian instance counts equal tiles_touched."""
    keys = keys[:m].view(np.uint64)
    vals = vals[:m].view(np.uint32)
    assert np.all(keys[1:] >= keys[:-1]), "keys not sorted"
    tile = (keys >> np.uint64(32)).astype(np.int64)
    dbits = (keys & np.uint64(0xFFFFFFFF)).astype(np.uint32)
    assert np.array_equal(dbits, recs["depth"].view(np.uint32)[vals]), "depth bits do not match the value"
    r = rect_of(recs)[vals]
    tx, ty = tile % tiles_x, tile // tiles_x
    assert np.all((tx >= r[:, 0]) & (tx < r[:, 2]) & (ty >= r[:, 1]) & (ty < r[:, 3])), "tile outside rect"
    counts = np.bincount(vals, minlength=len(recs))
    assert np.array_equal(counts, recs["tiles_touched"].astype(np.int64)), "instance count != tiles_touched"
    # ties: equal keys keep ascending id
    same = keys[1:] == keys[:-1]
    assert np.all(vals[1:][same] > vals[:-1][same]), "equal keys out of id order"
    rg = ranges.view(np.uint32).reshape(-1, 2).astype(np.int64)
    ne = rg[:, 1] > rg[:, 0]
    assert int((rg[:, 1] - rg[:, 0]).sum()) == m
    for t in np.nonzero(ne)[0][:: max(1, int(ne.sum()) // 2000)]:
        s, e = rg[t]
        assert np.all(tile[s:e] == t) and (s == 0 or tile[s - 1] < t) and (e == m or tile[e] > t)
    assert np.all(rg[~ne] == 0)
