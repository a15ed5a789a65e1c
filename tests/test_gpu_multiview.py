"""Several views of one scene in one persistent launch (gs_render_batch):
each view's outputs equal its own gs_render bit for bit, on a slab scene
whose occluding slab makes a few tiles far heavier than the rest."""

import numpy as np
import pytest
import torch

import paper_2509_25626_gb300 as gs
from synth import orbit_camera, slab_scene

pytestmark = pytest.mark.gpu


def test_multiview_batch_equals_single_views():
    sc = slab_scene(200_000, seed=21)
    st = gs.SceneTensors.from_scene(sc, "cuda")
    cams = [orbit_camera(k, 8, 4.0, 480, 270, arc=np.radians(40.0)) for k in range(8)]
    views = []
    for cam in cams:
        sp = gs.preprocess(st, cam)
        _, vals, ranges, m, _ = gs.sort(sp, st.n, cam, 1 << 23)
        views.append((cam, sp, vals, ranges, gs.render(sp, vals, ranges, cam)))
    lens = [int((r[:, 1] - r[:, 0]).max()) for _, _, _, r, _ in views]
    assert max(lens) > 20 * np.mean([float((r[:, 1] - r[:, 0]).float().mean()) for _, _, _, r, _ in views])
    outs = [tuple(torch.empty_like(t) for t in v[4]) for v in views]
    rb = gs.RenderBatch(8)
    rb.set_jobs([gs.BatchJob(sp, v, r, *o, c.width, c.height) for (c, sp, v, r, _), o in zip(views, outs)])
    rb.launch()
    torch.cuda.synchronize()
    for (cam, sp, vals, ranges, ref), out in zip(views, outs):
        for a, b in zip(out, ref):
            assert torch.equal(a, b)


@pytest.mark.parametrize("n_jobs", [64, 70])
def test_batch_job_table_sizes(n_jobs):
    """A batch of many small jobs (mixed sizes and backgrounds): up to 64 the
    kernel keeps the job table in shared memory, beyond it reads each item's
    job from device memory; both give every job its own gs_render output."""
    sc = slab_scene(20_000, seed=5)
    st = gs.SceneTensors.from_scene(sc, "cuda")
    sizes = [(48, 32), (33, 17), (64, 64), (16, 16), (80, 45)]
    jobs = []
    for k in range(n_jobs):
        w, h = sizes[k % len(sizes)]
        cam = orbit_camera(k % 8, 8, 4.0, w, h, arc=np.radians(40.0))
        bg = (0.1 * (k % 3), 0.2, 0.05 * (k % 5))
        sp = gs.preprocess(st, cam)
        _, vals, ranges, m, _ = gs.sort(sp, st.n, cam, 1 << 20)
        ref = gs.render(sp, vals, ranges, cam, bg)
        jobs.append((cam, bg, sp, vals, ranges, ref, tuple(torch.empty_like(t) for t in ref)))
    rb = gs.RenderBatch(n_jobs)
    rb.set_jobs([gs.BatchJob(sp, v, r, *o, c.width, c.height, bg) for c, bg, sp, v, r, _, o in jobs])
    rb.launch()
    torch.cuda.synchronize()
    for c, bg, sp, v, r, ref, out in jobs:
        for a, b in zip(out, ref):
            assert torch.equal(a, b)


def test_full_size_slab_views_sampled(oracle):
    """The load-imbalance workload at full size -- 6M Gaussians, half of them
    in the occluding slab, 3840x2160 -- with two of its views rendered in one
    gs_render_batch launch as the benchmark does: the batch equals each
    view's own frame bit for bit, the first view's sort has the properties a
    sort has at any size, and the tile rows through the slab (the longest
    lists) match the oracle.  The oracle sorts only the instances of those
    rows: each Gaussian's rectangle clipped to them leaves their tiles' lists
    and order unchanged."""
    from paper_2509_25626_gb300 import SPLAT_DTYPE
    from parity import (POS_EPS_E2E, TAU_ALPHA, TAU_T, ambiguous_gaussians, check_sorted_output, compare_images,
                        flip_tile_mask, rect_of)
    sc = slab_scene(6_000_000, seed=5)
    st = gs.SceneTensors.from_scene(sc, "cuda")
    cams = [orbit_camera(k, 8, 4.0, 3840, 2160, arc=np.radians(40.0)) for k in (0, 7)]
    rs = []
    for cam in cams:
        r = gs.Renderer(sc.n, cam.width, cam.height, 90_000_000)
        r.frame(st, cam)
        m, over = r.instances()
        assert not over
        rs.append((r, m))
    outs = [tuple(torch.empty_like(t) for t in (r.image, r.final_T, r.n_contrib)) for r, _ in rs]
    rb = gs.RenderBatch(2)
    rb.set_jobs([gs.BatchJob(r.splats, r.vals, r.ranges, *o, c.width, c.height) for c, (r, _), o in
                 zip(cams, rs, outs)])
    rb.launch()
    torch.cuda.synchronize()
    for (r, _), out in zip(rs, outs):
        for a, b in zip(out, (r.image, r.final_T, r.n_contrib)):
            assert torch.equal(a, b)

    cam, (r, m) = cams[0], rs[0]
    recs = r.splats.cpu().numpy().view(SPLAT_DTYPE).reshape(-1)[: sc.n]
    check_sorted_output(r.keys.cpu().numpy(), r.vals.cpu().numpy(), r.ranges.cpu().numpy(), m, recs, cam.tiles_x)
    lens = r.ranges.cpu().numpy().astype(np.int64)
    ty0, ty1 = 66, 68  # tile rows through the slab
    rows = (16 * ty0, 16 * ty1)
    band_lens = (lens[:, 1] - lens[:, 0]).reshape(cam.tiles_y, cam.tiles_x)[ty0:ty1]
    assert band_lens.max() > 50 * max(1.0, float((lens[:, 1] - lens[:, 0]).mean()))  # the heavy tiles

    pre = oracle.preprocess(sc, cam)
    clip = dict(pre)
    rect = pre["rect"].copy()
    rect[:, 1] = np.maximum(rect[:, 1], ty0)
    rect[:, 3] = np.minimum(rect[:, 3], ty1)
    keep = (pre["tiles"] > 0) & (rect[:, 3] > rect[:, 1])
    clip["rect"] = np.where(keep[:, None], rect, 0).astype(np.int32)
    clip["tiles"] = np.where(keep, (rect[:, 2] - rect[:, 0]) * (rect[:, 3] - rect[:, 1]), 0).astype(np.int32)
    srt = oracle.duplicate_sort(clip, cam)
    img = oracle.render(clip, srt, cam, tau_alpha=TAU_ALPHA, tau_T=TAU_T, rows=rows, pos_eps=POS_EPS_E2E)
    sl = slice(*rows)
    band = {k: (v[:, sl] if k == "color" else v[sl]) for k, v in img.items()}
    flips = np.nonzero((recs["tiles_touched"].astype(np.int64) != pre["tiles"]) |
                       np.any(rect_of(recs) != pre["rect"], axis=1))[0]
    assert np.all(ambiguous_gaussians(pre, cam)[flips]), "a rectangle flipped on a non-ambiguous Gaussian"
    amb = flip_tile_mask(recs, pre, flips, cam, rows=rows)
    rep = compare_images(outs[0][0].cpu().numpy()[:, sl], outs[0][1].cpu().numpy()[sl],
                         outs[0][2].cpu().numpy()[sl], band, exclude=amb, max_excluded_frac=0.03)
    print("slab full size", m, int(band_lens.max()), rep)
    # the same two views through the balanced render (long lists first and
    # heavy tiles split): the band at the same bar
    souts = [tuple(torch.empty_like(t) for t in o) for o in outs]
    rb = gs.RenderBatch(2)
    rb.set_jobs([gs.BatchJob(r.splats, r.vals, r.ranges, *so, c.width, c.height) for c, (r, _), so in
                 zip(cams, rs, souts)])
    params = gs.BalanceParams(heavy_len=4096, max_heavy_tiles=4096, budget=4096, max_split_tiles=4096,
                              max_chunks=32, chunk=1024)
    ws = gs.balance_workspace(params)
    rb.launch_balanced(params, ws)
    torch.cuda.synchronize()
    n_split = int(ws[:4].view(torch.int32).item())
    rep = compare_images(souts[0][0].cpu().numpy()[:, sl], souts[0][1].cpu().numpy()[sl],
                         souts[0][2].cpu().numpy()[sl], band, exclude=amb, max_excluded_frac=0.03)
    print("slab full size, split render", n_split, rep)


def _split_entries(ws, heavy_cap):
    """The tiles the balanced render split: (job, tile, begin, pos, end).
    The workspace holds a 256-byte header, the long-list queue, then these."""
    n = int(ws[:4].view(torch.int32).item())
    at = 256 + (4 * heavy_cap + 255) // 256 * 256
    ent = ws[at:at + 32 * max(n, 1)].view(torch.int32).reshape(-1, 8)[:n, :5].cpu().numpy()
    return n, ent


def _views(sc, cams, m_cap):
    st = gs.SceneTensors.from_scene(sc, "cuda")
    out = []
    for cam in cams:
        sp = gs.preprocess(st, cam)
        _, vals, ranges, m, _ = gs.sort(sp, st.n, cam, m_cap)
        out.append((cam, sp, vals, ranges, [t.clone() for t in gs.render(sp, vals, ranges, cam)]))
    return out


@pytest.mark.parametrize("cap,heavy", [(4096, 0), (3, 0), (4096, 1024)])
def test_split_render_matches_single_walk_and_oracle(oracle, cap, heavy):
    """gs_render_batch_balanced with a small budget (one round of 256
    splats), so that many tiles are split into chunks: tiles finished within
    the budget equal gs_render bit for bit; split tiles equal it up to the
    FP32 rounding of the regrouped products; every view matches the oracle
    at the parity bar.  cap = 3: the split queue holds only three tiles, the
    rest of the heavy tiles are walked whole by the block that started them.
    heavy = 1024: long lists are also started first."""
    from paper_2509_25626_gb300 import SPLAT_DTYPE
    from parity import POS_EPS_E2E, TAU_ALPHA, TAU_T, ambiguous_gaussians, compare_images, flip_tile_mask, rect_of
    sc = slab_scene(200_000, seed=21)
    cams = [orbit_camera(k, 8, 4.0, 480, 270, arc=np.radians(40.0)) for k in (0, 3, 7)]
    views = _views(sc, cams, 1 << 23)
    outs = [tuple(torch.empty_like(t) for t in v[4]) for v in views]
    rb = gs.RenderBatch(len(views))
    rb.set_jobs([gs.BatchJob(sp, v, r, *o, c.width, c.height) for (c, sp, v, r, _), o in zip(views, outs)])
    params = gs.BalanceParams(heavy_len=heavy, max_heavy_tiles=4096 if heavy else 0, budget=256,
                              max_split_tiles=cap, max_chunks=8, chunk=256)
    ws = gs.balance_workspace(params)
    rb.launch_balanced(params, ws)
    torch.cuda.synchronize()
    n, ent = _split_entries(ws, params.max_heavy_tiles if heavy else 0)
    assert n > 20  # many tiles ran out of budget
    split = {(int(j), int(t)) for j, t in ent[:min(n, cap), :2]}
    assert len(split) == min(n, cap)
    for jv, ((cam, sp, vals, ranges, ref), out) in enumerate(zip(views, outs)):
        tx = cam.tiles_x
        mask = np.zeros((cam.height, cam.width), bool)
        for j, t in split:
            if j == jv:
                ty, txx = divmod(t, tx)
                mask[16 * ty:16 * ty + 16, 16 * txx:16 * txx + 16] = True
        img, T, nc = (o.cpu().numpy() for o in out)
        rimg, rT, rnc = (r.cpu().numpy() for r in ref)
        assert np.array_equal(img[:, ~mask], rimg[:, ~mask]) and np.array_equal(T[~mask], rT[~mask])
        assert np.array_equal(nc[~mask], rnc[~mask])
        assert np.abs(img[:, mask] - rimg[:, mask]).max(initial=0) <= 5e-5
        assert np.abs(T[mask] - rT[mask]).max(initial=0) <= 5e-5
        pre, srt, ora = oracle.frame(sc, cam, (0.0, 0.0, 0.0), TAU_ALPHA, TAU_T, pos_eps=POS_EPS_E2E)
        recs = sp.cpu().numpy().view(SPLAT_DTYPE).reshape(-1)[: sc.n]
        flips = np.nonzero((recs["tiles_touched"].astype(np.int64) != pre["tiles"]) |
                           np.any(rect_of(recs) != pre["rect"], axis=1))[0]
        assert np.all(ambiguous_gaussians(pre, cam)[flips]), "a rectangle flipped on a non-ambiguous Gaussian"
        rep = compare_images(img, T, nc, ora, exclude=flip_tile_mask(recs, pre, flips, cam))
        print("split view", jv, "split tiles", int(mask.sum()) // 256, "rect flips", len(flips), rep)


@pytest.mark.parametrize("heavy_len,heavy_cap", [(1024, 4096), (64, 4096), (1024, 2)])
def test_long_lists_first_equals_single_views(heavy_len, heavy_cap):
    """gs_render_batch_balanced with long-list tiles started first and no
    splitting: only the order in which blocks take the tiles changes, so
    every view equals its own gs_render bit for bit -- also when nearly every
    tile qualifies (heavy_len 64) and when the queue overflows (capacity 2:
    the plain order is kept)."""
    sc = slab_scene(200_000, seed=21)
    cams = [orbit_camera(k, 8, 4.0, 480, 270, arc=np.radians(40.0)) for k in range(4)]
    views = _views(sc, cams, 1 << 23)
    outs = [tuple(torch.empty_like(t) for t in v[4]) for v in views]
    rb = gs.RenderBatch(len(views))
    rb.set_jobs([gs.BatchJob(sp, v, r, *o, c.width, c.height) for (c, sp, v, r, _), o in zip(views, outs)])
    params = gs.BalanceParams(heavy_len=heavy_len, max_heavy_tiles=heavy_cap, budget=0)
    ws = gs.balance_workspace(params)
    rb.launch_balanced(params, ws)
    torch.cuda.synchronize()
    n_heavy = int(ws[8:12].view(torch.int32).item())
    assert n_heavy > 0
    for (cam, sp, vals, ranges, ref), out in zip(views, outs):
        for a, b in zip(out, ref):
            assert torch.equal(a, b)
