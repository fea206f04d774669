"""Tile shapes, staging batches, persistent longest-first scheduling, the
CUDA-graph batched step and the autotuner, through the C ABI."""
import json
import os

import numpy as np
import pytest
import torch

import oracle
from paper_2501_18630_gb300 import _lib, autotune, batched, render, scenes
from tests import gpu_common as gc

pytestmark = pytest.mark.gpu

SHAPES = [(8, 4), (8, 8), (16, 8), (16, 16), (32, 16)]


@pytest.mark.parametrize("tw,th", SHAPES)
def test_bin_sort_bit_exact_every_tile_shape(tw, th):
    sc = scenes.config_scene(2, n=30_000)
    cams = [scenes.ring_camera(4.0, 20.0, 0.4, 333, 201), scenes.ring_camera(4.0, 20.0, 2.0, 160, 96)]
    opts = _lib.default_opts(tile_w=tw, tile_h=th)
    rast, _ = gc.rasterize(sc.planes, sc.n, sc.n_lobes, cams, opts=opts)
    K, ranges, vals = gc.sorted_pairs(rast)
    tiles, recs, oranges = oracle.bin_pairs(sc.planes, sc.n, sc.n_lobes, cams, tile_w=tw, tile_h=th,
                                            pitch=sc.pitch)
    assert K == len(recs)
    assert np.array_equal(ranges, oranges)
    assert np.array_equal(vals, recs)


def test_images_identical_across_shapes_batches_and_scheduling():
    """Every pixel composites the same Betas in the same order whatever the
    tiling, so the images are bit-identical; one configuration is also
    checked against the FP64 oracle."""
    sc = scenes.config_scene(3, n=40_000)
    cams = [scenes.ring_camera(4.0, 15.0, 0.0, 400, 300), scenes.ring_camera(4.0, 15.0, 1.3, 257, 129)]
    ref, _ = gc.rasterize(sc.planes, sc.n, sc.n_lobes, cams)
    ref_img = ref.color.cpu().numpy()
    ref_T = ref.T_final.cpu().numpy()
    for (tw, th) in SHAPES:
        for bs in (64, 256):
            for persist in (False, True):
                gc.ensure_built()
                planes = torch.from_numpy(sc.planes).cuda()
                r = render.Rasterizer(sc.n, sc.pitch, sc.n_lobes, cams,
                                      _lib.default_opts(tile_w=tw, tile_h=th, batch_s=bs), persistent=persist)
                r.forward(planes)
                torch.cuda.synchronize()
                assert np.array_equal(r.color.cpu().numpy(), ref_img), (tw, th, bs, persist)
                assert np.array_equal(r.T_final.cpu().numpy(), ref_T)
    xs, ys = scenes.sample_pixels(cams[1], 1024, seed=4)
    C, T, _, _ = oracle.render(sc.planes, sc.n, sc.n_lobes, cams[1], xs, ys)
    assert np.abs(gc.image(ref, 1)[:, ys, xs].T - C).max() <= gc.IMG_TOL


def test_persistent_gradients_match_default():
    sc = scenes.config_scene(3, n=40_000)
    cams = [scenes.ring_camera(4.0, 15.0, 0.7, 320, 240)]
    tgt = torch.from_numpy(scenes.target_images(cams, seed=2)[0].reshape(-1)).cuda()
    grads = []
    # the default 16x16 and every other tile shape but 8x4 run the pixel-pair
    # kernels; 8x4 the one-pixel-per-lane ones, a direct cross-check of the two
    for opts, persist in ((None, False), (_lib.default_opts(tile_w=32, tile_h=16, batch_s=128), True),
                          (_lib.default_opts(tile_w=8, tile_h=8, batch_s=64), True),
                          (_lib.default_opts(tile_w=16, tile_h=8, batch_s=128), False),
                          (_lib.default_opts(tile_w=16, tile_h=8, batch_s=128), True),
                          (_lib.default_opts(tile_w=16, tile_h=8, batch_s=64), False),
                          (_lib.default_opts(tile_w=8, tile_h=4, batch_s=64), False),
                          (_lib.default_opts(tile_w=8, tile_h=4, batch_s=128), True)):
        gc.ensure_built()
        planes = torch.from_numpy(sc.planes).cuda()
        r = render.Rasterizer(sc.n, sc.pitch, sc.n_lobes, cams, opts, persistent=persist)
        r.forward(planes)
        _, d = r.l1_loss(tgt)
        grads.append(r.backward(planes, d).cpu().numpy()[:, :sc.n].astype(np.float64))
    for g in grads[1:]:
        # atomics sum in a different order: float-rounding differences only
        scale = np.abs(grads[0]).max(axis=1, keepdims=True) + 1e-30
        assert np.max(np.abs(g - grads[0]) / scale) < 1e-4


def test_graph_replay_matches_eager_step():
    sc = scenes.config_scene(4, n=60_000, n_views=8)
    cams = sc.cameras[::2]
    gc.ensure_built()
    planes = torch.from_numpy(sc.planes).cuda()
    tgt = torch.from_numpy(np.concatenate([t.reshape(-1) for t in scenes.target_images(cams, seed=8)])).cuda()
    step = batched.BatchedStep(planes, sc.n, sc.n_lobes, cams, tgt)
    step.step()
    k = step.check()
    assert k > 0
    img_g = step.rast.color.clone()
    loss_g = step.loss.clone()
    grad_g = step.grad.clone()
    step.step()                                    # replay again: same results
    torch.cuda.synchronize()
    assert torch.equal(step.rast.color, img_g)
    # eager reference through a plain rasterizer
    r = render.Rasterizer(sc.n, sc.pitch, sc.n_lobes, cams)
    r.forward(planes)
    loss_e, d = r.l1_loss(tgt)
    grad_e = r.backward(planes, d)
    torch.cuda.synchronize()
    assert torch.equal(r.color, img_g)
    assert torch.allclose(loss_e, loss_g, rtol=1e-6, atol=0)
    scale = grad_e.abs().amax(dim=1, keepdim=True) + 1e-30
    assert float(((grad_g - grad_e).abs() / scale).max()) < 1e-4


def test_graph_capacity_overflow_recaptures():
    sc = scenes.config_scene(1, n=4096)
    gc.ensure_built()
    planes = torch.from_numpy(sc.planes).cuda()
    cams = sc.cameras
    tgt = torch.from_numpy(scenes.target_images(cams, seed=1)[0].reshape(-1)).cuda()
    step = batched.BatchedStep(planes, sc.n, sc.n_lobes, cams, tgt)
    step.step()
    k0 = step.check()
    # scale every Beta up 4x: the pair count outgrows the sized buffers
    planes[3:6] += float(np.log(4.0))
    step.step()
    k1 = step.check()                     # grows the buffers, recaptures, replays
    assert k1 > k0 and step.rast.cap >= k1
    r = render.Rasterizer(sc.n, sc.pitch, sc.n_lobes, cams)
    r.forward(planes)
    torch.cuda.synchronize()
    assert torch.equal(r.color, step.rast.color)


def test_autotuner_times_candidates_and_caches(tmp_path, monkeypatch):
    monkeypatch.setenv("BETA_AUTOTUNE_CACHE", str(tmp_path / "tune.json"))
    sc = scenes.config_scene(3, n=20_000)
    cams = [scenes.ring_camera(4.0, 15.0, 0.0, 320, 240)]
    gc.ensure_built()
    planes = torch.from_numpy(sc.planes).cuda()
    tgt = torch.from_numpy(scenes.target_images(cams, seed=3)[0].reshape(-1)).cuda()
    # the last candidate runs the raster forward and backward as two launches
    cands = [(16, 16, 256, True), (16, 8, 64, False), (16, 8, 64, False, False)]
    best, times = autotune.tune(planes, sc.n, sc.n_lobes, cams, tgt, candidates=cands, reps=2)
    assert best in cands and set(times) == set(cands) and all(t > 0 for t in times.values())
    d = json.load(open(tmp_path / "tune.json"))
    assert len(d) == 1 and list(d.values())[0]["best"] == list(best)
    best2, _ = autotune.tune(planes, sc.n, sc.n_lobes, cams, tgt, candidates=cands)
    assert best2 == best
    # restricted to two launches, every candidate is timed that way
    _, t3 = autotune.tune(planes, sc.n, sc.n_lobes, cams, tgt, candidates=cands[:2], reps=1, fused=False)
    assert set(t3) == {(16, 16, 256, True, False), (16, 8, 64, False, False)}


def test_view_split_gradients_sum_to_full_batch():
    """The data-parallel split over views: views {0..7} and {8..15} rendered
    as two batched steps, their gradients summed, equal the 16-view step's
    gradient (1e-4 of each plane's largest value) and their losses are the
    16-view step's losses.  This is what the gradient all-reduce of the
    multi-GPU path relies on."""
    sc = scenes.config_scene(3, n=200_000)
    cams = scenes.ring_cameras(16, 4.0, 15.0, [(640, 360)] * 16)
    tg = scenes.target_images(cams, seed=21)
    gc.ensure_built()
    planes = torch.from_numpy(sc.planes).cuda()
    opts = _lib.default_opts(tile_w=16, tile_h=8, batch_s=128)

    def run(vs):
        t = torch.from_numpy(np.concatenate([tg[v].reshape(-1) for v in vs])).cuda()
        st = batched.BatchedStep(planes, sc.n, sc.n_lobes, [cams[v] for v in vs], t, opts=opts, persistent=False)
        st.step()
        st.check()
        torch.cuda.synchronize()
        return st.grad.cpu().numpy()[:, :sc.n].astype(np.float64), st.loss.cpu().numpy()

    g_all, l_all = run(list(range(16)))
    g_a, l_a = run(list(range(8)))
    g_b, l_b = run(list(range(8, 16)))
    assert np.array_equal(np.concatenate([l_a, l_b]), l_all)
    scale = np.abs(g_all).max(axis=1, keepdims=True) + 1e-30
    assert np.all(np.abs(g_all).max(axis=1) > 0)
    assert np.max(np.abs(g_a + g_b - g_all) / scale) < 1e-4


@pytest.mark.parametrize("tw,th,bs,persist", [(16, 8, 128, False), (16, 16, 256, True), (8, 8, 64, False),
                                              (32, 16, 128, True)])
def test_hit_masks_give_the_same_results(tw, th, bs, persist):
    """With the hit-mask buffer the forward keeps, per pixel, which Betas may
    cover it and the backward reads that instead of redoing its cover pass:
    images, T and n_contrib bit for bit, gradients within 1e-4 of each
    plane's largest value (atomics add in another order).  A buffer too short
    for the whole list (the backward recomputes the rest) gives the same."""
    sc = scenes.config_scene(3, n=60_000)
    cams = [scenes.ring_camera(4.0, 15.0, 0.7, 333, 201), scenes.ring_camera(4.0, 15.0, 2.2, 160, 97)]
    tgt = torch.from_numpy(np.concatenate([t.reshape(-1) for t in scenes.target_images(cams, seed=5)])).cuda()
    gc.ensure_built()
    planes = torch.from_numpy(sc.planes).cuda()
    opts = _lib.default_opts(tile_w=tw, tile_h=th, batch_s=bs)
    out = []
    for mode in ("none", "full", "short"):
        r = render.Rasterizer(sc.n, sc.pitch, sc.n_lobes, cams, opts, persistent=persist,
                              hit_masks=mode != "none")
        r.forward(planes)
        if mode == "short":
            r.hit_masks = r.hit_masks[: r.hit_masks.numel() // 3]
            r.raster_fwd(planes)
        _, d = r.l1_loss(tgt)
        g = r.backward(planes, d)
        torch.cuda.synchronize()
        out.append((r.color.clone(), r.T_final.clone(), r.n_contrib.clone(), g.cpu().numpy()[:, :sc.n]))
    (c0, t0, n0, g0) = out[0]
    scale = np.abs(g0).max(axis=1, keepdims=True) + 1e-30
    for (c, t, n_, g) in out[1:]:
        assert torch.equal(c, c0) and torch.equal(t, t0) and torch.equal(n_, n0)
        assert np.max(np.abs(g - g0) / scale) < 1e-4


def test_projection_backward_in_chunks_equals_whole():
    """The projection backward over primitive ranges (pointers offset by the
    range start, the full pitch kept) gives the whole call's gradients bit
    for bit from the same 2D gradients; the batched step with the projection
    backward run in chunks after the replay (the multi-GPU overlap path, one
    rank here) matches the step with it inside the graph."""
    sc = scenes.config_scene(3, n=50_003)
    sc = scenes.Scene(planes=np.ascontiguousarray(sc.planes), n=50_003, n_lobes=sc.n_lobes, cameras=sc.cameras)
    cams = [scenes.ring_camera(4.0, 15.0, 0.7, 320, 240), scenes.ring_camera(4.0, 15.0, 2.0, 200, 150)]
    tgt = torch.from_numpy(np.concatenate([t.reshape(-1) for t in scenes.target_images(cams, seed=12)])).cuda()
    gc.ensure_built()
    planes = torch.from_numpy(sc.planes).cuda()
    r = render.Rasterizer(sc.n, sc.pitch, sc.n_lobes, cams)
    r.forward(planes)
    _, d = r.l1_loss(tgt)
    r.raster_bwd(planes, d)
    saved = r.grad2d.clone()
    g_whole = torch.zeros_like(planes)
    r.project_bwd(planes, g_whole)
    r.grad2d.copy_(saved)
    g_parts = torch.zeros_like(planes)
    from paper_2501_18630_gb300 import distributed
    for c0, c1 in distributed.chunk_ranges(sc.n, 7001):
        r.project_bwd(planes, g_parts, c0, c1)
    torch.cuda.synchronize()
    assert torch.equal(g_whole, g_parts)
    assert bool((r.grad2d == 0).all())                     # every consumed slot cleared
    opts = _lib.default_opts(tile_w=16, tile_h=8, batch_s=128)
    a = batched.BatchedStep(planes, sc.n, sc.n_lobes, cams, tgt, opts=opts, persistent=False)
    a.step()
    a.check()
    b = batched.BatchedStep(planes, sc.n, sc.n_lobes, cams, tgt, opts=opts, persistent=False,
                            graph_project_bwd=False)
    b.step()
    b.project_bwd_reduced(chunk=9000)
    b.check()
    torch.cuda.synchronize()
    ga, gb = a.grad.cpu().numpy()[:, :sc.n], b.grad.cpu().numpy()[:, :sc.n]
    scale = np.abs(ga).max(axis=1, keepdims=True) + 1e-30
    assert np.max(np.abs(ga - gb) / scale) < 1e-4
