"""Full-size workloads beyond the benchmark's: 3M Betas over views of mixed
resolution, and 6M Betas over eight 3840x2160 views in one captured step
under a stated HBM budget."""
import numpy as np
import pytest
import torch

import oracle
from paper_2501_18630_gb300 import batched, scenes
from tests import gpu_common as gc

pytestmark = pytest.mark.gpu

HBM_BUDGET_BYTES = 24 * 1024 ** 3


def test_3m_betas_mixed_resolution_views():
    sc = scenes.config_scene(4)                          # 3M Betas, 16 mixed views
    cams = sc.cameras[::4]                               # one view of each resolution
    rast, _ = gc.rasterize(sc.planes, sc.n, sc.n_lobes, cams)
    K, ranges, vals = gc.sorted_pairs(rast)
    tiles, recs, oranges = oracle.bin_pairs(sc.planes, sc.n, sc.n_lobes, cams, pitch=sc.pitch)
    assert K == len(recs) and np.array_equal(ranges, oranges) and np.array_equal(vals, recs)
    for v in (0, 3):
        xs, ys = scenes.sample_pixels(cams[v], 512, seed=40 + v, full_tiles=1)
        C, T, _, _ = oracle.render(sc.planes, sc.n, sc.n_lobes, cams[v], xs, ys)
        assert np.abs(gc.image(rast, v)[:, ys, xs].T - C).max() <= gc.IMG_TOL


def test_6m_betas_eight_4k_views_in_budget():
    sc = scenes.config_scene(5)                          # 6M Betas, 8 views of 3840x2160
    gc.ensure_built()
    torch.cuda.empty_cache()
    torch.cuda.reset_peak_memory_stats()
    base = torch.cuda.memory_allocated()
    planes = torch.from_numpy(sc.planes).cuda()
    tgt = torch.from_numpy(np.concatenate([t.reshape(-1) for t in scenes.target_images(sc.cameras, seed=6)])).cuda()
    step = batched.BatchedStep(planes, sc.n, sc.n_lobes, sc.cameras, tgt)
    step.step()
    k = step.check()
    torch.cuda.synchronize()
    peak = torch.cuda.max_memory_allocated() - base
    assert k > sc.n and peak <= HBM_BUDGET_BYTES, (k, peak / 2 ** 30)
    assert torch.isfinite(step.loss).all() and torch.isfinite(step.grad).all()
    for v in (0, 5):
        xs, ys = scenes.sample_pixels(sc.cameras[v], 256, seed=50 + v)
        C, T, _, _ = oracle.render(sc.planes, sc.n, sc.n_lobes, sc.cameras[v], xs, ys)
        img = step.rast.image(step.rast.color, v).cpu().numpy().astype(np.float64)
        assert np.abs(img[:, ys, xs].T - C).max() <= gc.IMG_TOL


def test_1m_betas_sixteen_views_benchmark_configuration():
    """The benchmark's own step: 1M Betas, 16 ring views of 1920x1080, 16x8
    tiles, 128-record batches, one CTA per tile, captured and replayed.  Two
    views' binning equals the oracle's bit for bit (a view's lists are the
    view's own); sampled pixels of two views (including whole tiles) equal
    the FP64 oracle; the loss and gradients are finite."""
    from paper_2501_18630_gb300 import _lib
    sc = scenes.config_scene(3)
    cams = sc.cameras
    gc.ensure_built()
    planes = torch.from_numpy(sc.planes).cuda()
    tgt = torch.from_numpy(np.concatenate([t.reshape(-1) for t in scenes.target_images(cams, seed=77)])).cuda()
    step = batched.BatchedStep(planes, sc.n, sc.n_lobes, cams, tgt,
                               opts=_lib.default_opts(tile_w=16, tile_h=8, batch_s=128), persistent=False)
    step.step()
    k = step.check()
    torch.cuda.synchronize()
    r = step.rast
    ranges = r.ranges.cpu().numpy().view(np.uint32)
    vals = r.pair_vals[:k].cpu().numpy().view(np.uint32)
    for v in (0, 9):
        _, recs, oranges = oracle.bin_pairs(sc.planes, sc.n, sc.n_lobes, [cams[v]], tile_w=16, tile_h=8,
                                            pitch=sc.pitch)
        t0 = sum(int(np.prod(oracle.n_tiles(c, 16, 8))) for c in cams[:v])
        t1 = t0 + len(oranges) - 1
        lo = ranges[t0]
        assert np.array_equal(ranges[t0:t1 + 1] - lo, oranges)
        assert np.array_equal(vals[lo:ranges[t1]] - v * sc.pitch, recs)
        xs, ys = scenes.sample_pixels(cams[v], 384, seed=60 + v, full_tiles=1)
        C, T, _, _ = oracle.render(sc.planes, sc.n, sc.n_lobes, cams[v], xs, ys)
        img = r.image(r.color, v).cpu().numpy().astype(np.float64)
        assert np.abs(img[:, ys, xs].T - C).max() <= gc.IMG_TOL
    assert torch.isfinite(step.loss).all() and torch.isfinite(step.grad).all()
    assert float(step.grad.abs().max()) > 0.0
