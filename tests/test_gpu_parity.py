"""CUDA path vs FP64 oracle, through the C ABI.

Bars: tile assignment and key order bit-exact; image within 2e-5 absolute per
channel; gradients within 1e-3 relative of central finite differences of the
oracle on every (primitive, parameter-group) block of norm > 1e-6.
"""
import math

import numpy as np
import pytest
import torch

import oracle
from paper_2501_18630_gb300 import _lib, render, scenes
from tests import gpu_common as gc
from tests.helpers import planes_of, prim

pytestmark = pytest.mark.gpu


# --------------------------------------------------------------------------
# step 1: projection records
# --------------------------------------------------------------------------

@pytest.mark.parametrize("cfg,n,views", [(1, 4096, [0]), (3, 20000, [0, 5]), (2, 20000, [0])])
def test_project_records_match_oracle(cfg, n, views):
    sc = scenes.config_scene(cfg, n=n)
    cams = [sc.cameras[v] for v in views]
    rast, _ = gc.rasterize(sc.planes, sc.n, sc.n_lobes, cams)
    rec, rects, keys, tiles = gc.proj_arrays(rast, with_tiles=True)
    for v, cam in enumerate(cams):
        pr = oracle.project(sc.planes, sc.n, sc.n_lobes, cam)
        orects, okeys, obinned, otiles = oracle.rule_rects(sc.planes, sc.n, sc.n_lobes, cam, with_tiles=True)
        binned = (rects[v, :n, 0] <= rects[v, :n, 1]) & (rects[v, :n, 2] <= rects[v, :n, 3])
        assert np.array_equal(binned, obinned > 0)
        b = np.nonzero(binned)[0]
        assert np.array_equal(rects[v, b], orects[b])
        assert np.array_equal(keys[v, b], okeys[b])
        assert np.array_equal(tiles[v, b], otiles[b])          # rule B2, bit for bit
        assert np.all(keys[v, np.nonzero(~binned)[0]] == 0xFFFFFFFF)
        r = rec[v, b].astype(np.float64)
        mu2 = np.stack([r[:, 0] + 0.5 - r[:, 2], r[:, 1] + 0.5 - r[:, 3]], -1)
        assert np.abs(mu2 - pr["mu2"][b]).max() < 1e-5
        p, q1, q2 = r[:, 4], r[:, 5], r[:, 6]
        Q = np.stack([p * p + q2 * q2, q1 * q2, q1 * q1], -1)
        Qo = pr["conic"][b]
        scale = np.abs(Qo).max(1, keepdims=True)
        assert np.abs(Q - Qo).max() / 1 < 1 and np.max(np.abs(Q - Qo) / scale) < 2e-4
        assert np.max(np.abs(r[:, 7] - pr["beta"][b]) / pr["beta"][b]) < 2e-6
        assert np.max(np.abs(np.exp2(r[:, 8]) - pr["o"][b]) / pr["o"][b]) < 2e-6
        assert np.abs(r[:, 9:12] - pr["color"][b]).max() < 2e-6


# --------------------------------------------------------------------------
# step 2: binning + per-tile list sort, bit-exact
# --------------------------------------------------------------------------

def _check_bins(sc, cams):
    rast, _ = gc.rasterize(sc.planes, sc.n, sc.n_lobes, cams)
    K, ranges, vals = gc.sorted_pairs(rast)
    tiles, recs, oranges = oracle.bin_pairs(sc.planes, sc.n, sc.n_lobes, cams, pitch=sc.pitch)
    assert K == len(recs)
    assert np.array_equal(ranges, oranges)
    assert np.array_equal(vals, recs)
    return K


@pytest.mark.parametrize("cfg,n", [(1, 4096), (2, 200_000), (3, 1_000_000)])
def test_bin_sort_bit_exact_full_size(cfg, n):
    sc = scenes.config_scene(cfg, n=n)
    K = _check_bins(sc, sc.cameras[:1])
    assert K > n // 4


def test_bin_sort_bit_exact_mixed_view_batch():
    sc = scenes.config_scene(4, n=60_000, n_views=16)
    K = _check_bins(sc, sc.cameras[::3])   # 6 views of mixed resolution
    assert K > 0


@pytest.mark.parametrize("cfg,n_views,tile,bits", [(3, 16, 16, 17), (5, 8, 16, 18), (5, 8, 8, 20)])
def test_bin_sort_bit_exact_wide_tile_ids(cfg, n_views, tile, bits):
    """Many tiles (17-20-bit global tile ids: up to 1M counters and lists,
    hundreds of scan blocks chained by look-back): lists equal the oracle's
    bit for bit."""
    sc = scenes.config_scene(cfg, n=20_000, n_views=n_views)
    opts = _lib.default_opts(tile_w=tile, tile_h=tile)
    total = sum(((c.width + tile - 1) // tile) * ((c.height + tile - 1) // tile) for c in sc.cameras)
    assert (total - 1).bit_length() == bits
    rast, _ = gc.rasterize(sc.planes, sc.n, sc.n_lobes, sc.cameras, opts=opts)
    K, ranges, vals = gc.sorted_pairs(rast)
    _, recs, oranges = oracle.bin_pairs(sc.planes, sc.n, sc.n_lobes, sc.cameras, tile_w=tile, tile_h=tile,
                                        pitch=sc.pitch)
    assert K == len(recs) and K > 0
    assert np.array_equal(ranges, oranges)
    assert np.array_equal(vals, recs)


def test_bin_sort_ragged_sizes():
    for n in (1, 3, 4095, 4096, 4097, 9000):
        sc = scenes.config_scene(1, n=n, seed=11)
        cam = scenes.pinhole(*scenes.look_at((0.0, 0.0, -3.0)), 37, 53)
        _check_bins(sc, [cam])


@pytest.mark.parametrize("n,pitch", [(1001, 1004), (4097, 4100), (300, 300)])
def test_bin_sort_pitch_not_a_multiple_of_the_warp(n, pitch):
    """A pitch that is a multiple of 4 but not of 32 (the last projection warp
    is partial): records, rule B2 tile masks and lists equal the oracle's."""
    base = scenes.config_scene(3, n=n, seed=13)
    planes = np.zeros((base.planes.shape[0], pitch), np.float32)
    planes[:, :n] = base.planes[:, :n]
    planes[6, n:] = 1.0
    cams = [scenes.ring_camera(4.0, 15.0, 0.3, 333, 201), scenes.ring_camera(4.0, 15.0, 1.9, 150, 90)]
    sc = scenes.Scene(planes=planes, n=n, n_lobes=base.n_lobes, cameras=cams, name="ragged pitch")
    assert _check_bins(sc, cams) > 0


def test_bin_sort_lists_longer_than_one_shared_memory_pass():
    """60k small Betas on a 24x20 image: lists of ~12k (sorted in 4096-item
    chunks and merged through global memory), ~3.5k, ~1.3k and ~500 items (the
    CTA sorts of 16, 8 and 4 items a thread) equal the oracle's."""
    sc = scenes.config_scene(1, n=60_000, seed=12)
    cam = scenes.pinhole(*scenes.look_at((0.0, 0.0, -3.0)), 24, 20)
    rast, _ = gc.rasterize(sc.planes, sc.n, sc.n_lobes, [cam])
    K, ranges, vals = gc.sorted_pairs(rast)
    _, recs, oranges = oracle.bin_pairs(sc.planes, sc.n, sc.n_lobes, [cam], pitch=sc.pitch)
    lens = np.diff(oranges)
    assert lens.max() > 2 * 4096 and ((lens > 512) & (lens <= 1024)).any()
    assert np.array_equal(ranges, oranges)
    assert np.array_equal(vals, recs)


def test_bin_sort_equal_depth_keys_keep_record_order():
    """Primitives repeated verbatim have equal depth keys in every tile they
    share: the lists hold them in record order, as the oracle's stable sort."""
    base = scenes.config_scene(1, n=700, seed=5)
    reps = 4
    n = base.n * reps
    planes = np.zeros((base.planes.shape[0], scenes.round_pitch(n)), np.float32)
    for r in range(reps):
        planes[:, r * base.n:(r + 1) * base.n] = base.planes[:, :base.n]
    sc = scenes.Scene(planes=planes, n=n, n_lobes=base.n_lobes, cameras=base.cameras, name="repeated")
    assert _check_bins(sc, sc.cameras) > 0


# --------------------------------------------------------------------------
# step 3: images
# --------------------------------------------------------------------------

def _compare_pixels(rast, v, sc, cam, xs, ys, tol=gc.IMG_TOL, **opts):
    """Image and T within tol of the FP64 oracle; the last contributor (from
    n_contrib) equal to the oracle's at every pixel, except where a support
    boundary or early-termination decision legitimately differs (each such
    pixel is checked individually)."""
    C, T, last, _ = oracle.render(sc.planes, sc.n, sc.n_lobes, cam, xs, ys, **opts)
    img = gc.image(rast, v)
    Tg = rast.plane(rast.T_final, v).cpu().numpy().astype(np.float64)
    err = np.abs(img[:, ys, xs].T - C)
    terr = np.abs(Tg[ys, xs] - T)
    lg = gc.last_ids(rast, v, sc.pitch)[ys, xs]
    assert err.max() <= tol, (err.max(), np.unravel_index(err.argmax(), err.shape))
    assert terr.max() <= tol, terr.max()
    pr = oracle.project(sc.planes, sc.n, sc.n_lobes, cam, **{k: w for k, w in opts.items()
                                                             if k in ("blur_eps", "b_lo", "b_hi")})
    bad, n_mism = gc.unexplained_last_mismatches(lg, last, T, xs, ys, pr)
    assert len(bad) == 0, (len(bad), n_mism, [(int(xs[k]), int(ys[k]), int(lg[k]), int(last[k])) for k in bad[:8]])
    return err.max()


def test_image_full_frame_4096_betas_256():
    sc = scenes.config_scene(1)
    cam = sc.cameras[0]
    rast, _ = gc.rasterize(sc.planes, sc.n, sc.n_lobes, [cam])
    ys, xs = np.mgrid[0:cam.height, 0:cam.width]
    _compare_pixels(rast, 0, sc, cam, xs.reshape(-1).astype(np.int32), ys.reshape(-1).astype(np.int32))


@pytest.mark.parametrize("cfg", [2, 3])
def test_image_sampled_full_size(cfg):
    """200k Betas at 1297x840 and 1M Betas at 1920x1080: 4096 seeded pixels
    plus 4 whole tiles, rendered at full size in the benchmark configuration."""
    sc = scenes.config_scene(cfg)
    cam = sc.cameras[0]
    rast, _ = gc.rasterize(sc.planes, sc.n, sc.n_lobes, [cam])
    xs, ys = scenes.sample_pixels(cam, 4096, seed=100 + cfg, full_tiles=4)
    _compare_pixels(rast, 0, sc, cam, xs, ys)


def test_image_batch_equals_single_views():
    sc = scenes.config_scene(4, n=50_000, n_views=8)
    cams = sc.cameras[::2]
    rast, _ = gc.rasterize(sc.planes, sc.n, sc.n_lobes, cams)
    for v, cam in enumerate(cams):
        one, _ = gc.rasterize(sc.planes, sc.n, sc.n_lobes, [cam])
        assert np.array_equal(gc.image(rast, v), gc.image(one, 0))
        xs, ys = scenes.sample_pixels(cam, 512, seed=v)
        _compare_pixels(rast, v, sc, cam, xs, ys)


def test_image_colour_modes_and_blur():
    sc = scenes.config_scene(1, n=2048)
    cam = scenes.pinhole(*scenes.look_at((0.0, 0.0, -3.0)), 96, 64)
    ys, xs = np.mgrid[0:cam.height, 0:cam.width]
    xs, ys = xs.reshape(-1).astype(np.int32), ys.reshape(-1).astype(np.int32)
    for mode, blur in ((1, 0.0), (2, 0.0), (0, 0.3)):
        rast, _ = gc.rasterize(sc.planes, sc.n, sc.n_lobes, [cam],
                               opts=_lib.default_opts(color_mode=mode, blur_eps=blur))
        C, T, _, _ = oracle.render(sc.planes, sc.n, sc.n_lobes, cam, xs, ys, color_mode=mode, blur_eps=blur)
        assert np.abs(gc.image(rast, 0)[:, ys, xs].T - C).max() <= gc.IMG_TOL


@pytest.mark.parametrize("tile,batch,persistent", [((16, 8), 128, False), ((16, 8), 128, True),
                                                    ((8, 8), 64, False), ((32, 16), 256, True),
                                                    ((16, 16), 256, False)])
def test_last_contributor_every_tile_shape(tile, batch, persistent):
    """n_contrib (1 + position in the tile's own list) names the oracle's last
    contributor at every pixel of two ragged views under every tile shape,
    batch and schedule; the few pixels where it differs are each a support
    boundary or early-termination decision."""
    sc = scenes.config_scene(3, n=40_000)
    cams = [scenes.ring_camera(4.0, 15.0, 0.7, 333, 201), scenes.ring_camera(4.0, 15.0, 2.2, 160, 97)]
    gc.ensure_built()
    planes = torch.from_numpy(sc.planes).cuda()
    rast = render.Rasterizer(sc.n, sc.pitch, sc.n_lobes, cams,
                             _lib.default_opts(tile_w=tile[0], tile_h=tile[1], batch_s=batch), persistent=persistent)
    rast.forward(planes)
    torch.cuda.synchronize()
    for v, cam in enumerate(cams):
        ys, xs = np.mgrid[0:cam.height, 0:cam.width]
        _compare_pixels(rast, v, sc, cam, xs.reshape(-1).astype(np.int32), ys.reshape(-1).astype(np.int32))


# --------------------------------------------------------------------------
# decomposition modes (Sec. 4.3): geometry mask on b, diffuse / specular colour
# --------------------------------------------------------------------------

@pytest.mark.parametrize("b_lo,b_hi", [(-math.inf, 0.0), (0.0, math.inf), (-0.3, 0.4)])
def test_geometry_mask_binning_and_image(b_lo, b_hi):
    """Only primitives with b_lo <= b < b_hi are binned (bit-exact against the
    oracle's masked lists) and rendered (within 2e-5 of the masked oracle)."""
    sc = scenes.config_scene(2, n=60_000)
    cams = [scenes.ring_camera(4.0, 20.0, 0.4, 416, 300)]
    opts = _lib.default_opts(b_lo=b_lo, b_hi=b_hi)
    rast, _ = gc.rasterize(sc.planes, sc.n, sc.n_lobes, cams, opts=opts)
    K, ranges, vals = gc.sorted_pairs(rast)
    _, recs, oranges = oracle.bin_pairs(sc.planes, sc.n, sc.n_lobes, cams, pitch=sc.pitch, b_lo=b_lo, b_hi=b_hi)
    _, recs_all, _ = oracle.bin_pairs(sc.planes, sc.n, sc.n_lobes, cams, pitch=sc.pitch)
    assert 0 < K == len(recs) < len(recs_all)
    assert np.array_equal(ranges, oranges) and np.array_equal(vals, recs)
    b = sc.planes[11, :sc.n]
    kept = (b >= np.float32(b_lo)) & (b < np.float32(b_hi))
    assert np.all(kept[np.unique(recs)])
    cam = cams[0]
    ys, xs = np.mgrid[0:cam.height, 0:cam.width]
    _compare_pixels(rast, 0, sc, cam, xs.reshape(-1).astype(np.int32), ys.reshape(-1).astype(np.int32),
                    b_lo=b_lo, b_hi=b_hi)


# --------------------------------------------------------------------------
# edge cases
# --------------------------------------------------------------------------

def test_empty_and_culled_scenes_render_background():
    cam = scenes.pinhole(*scenes.look_at((0.0, 0.0, -3.0)), 40, 24)
    cam.bg = (0.25, 0.5, 0.75)
    sc = scenes.config_scene(1, n=64)
    # every primitive behind the camera
    P = sc.planes.copy()
    P[2, :64] = -10.0
    for planes, n in ((sc.planes, 0), (P, 64)):
        rast, _ = gc.rasterize(planes, n, sc.n_lobes, [cam])
        st, K = rast.device_status()
        assert st == 0 and K == 0
        img = gc.image(rast, 0)
        assert np.allclose(img, np.array(cam.bg)[:, None, None].astype(np.float32))
        assert np.all(rast.T_final.cpu().numpy() == 1.0)


def test_non_finite_primitives_are_culled():
    sc = scenes.config_scene(1, n=512)
    cam = scenes.pinhole(*scenes.look_at((0.0, 0.0, -3.0)), 64, 64)
    P = sc.planes.copy()
    P[0, 3] = np.nan
    P[4, 7] = np.inf
    P[16, 9] = -np.inf     # a lobe parameter
    rast, _ = gc.rasterize(P, sc.n, sc.n_lobes, [cam])
    rec, rects, keys = gc.proj_arrays(rast)
    for i in (3, 7, 9):
        assert keys[0, i] == 0xFFFFFFFF
    ys, xs = np.mgrid[0:64, 0:64]
    _compare_pixels(rast, 0, scenes.Scene(P, sc.n, sc.n_lobes, [cam]), cam,
                    xs.reshape(-1).astype(np.int32), ys.reshape(-1).astype(np.int32))


def test_tiny_and_ragged_images_and_huge_splat():
    p_big = prim(mu=(0.0, 0.0, 1.0), scale=(0.8, 0.7, 0.6), opacity=0.6, b=0.2)
    p_small = prim(mu=(0.01, 0.0, 3.0), scale=(0.001, 0.002, 0.001), opacity=0.9, b=1.5)
    P = planes_of([p_small, p_big])
    for (w, h) in ((1, 1), (17, 33), (300, 7)):
        cam = scenes.pinhole(np.eye(3, dtype=np.float32), np.zeros(3, np.float32), w, h)
        rast, _ = gc.rasterize(P, 2, 0, [cam])
        ys, xs = np.mgrid[0:h, 0:w]
        sc = scenes.Scene(P, 2, 0, [cam])
        _compare_pixels(rast, 0, sc, cam, xs.reshape(-1).astype(np.int32), ys.reshape(-1).astype(np.int32))


def test_capacity_overflow_reports_and_recovers():
    sc = scenes.config_scene(1, n=4096)
    cam = sc.cameras[0]
    rast, planes = gc.rasterize(sc.planes, sc.n, sc.n_lobes, [cam], cap=100, check=False)
    st, K = rast.device_status()
    assert st == _lib.BETA_ERR_CAPACITY and K > 100
    # raster kernels skip work after a non-zero status; the retrying forward recovers
    rast.forward(planes, check_capacity=True)
    st2, K2 = rast.device_status()
    assert st2 == 0 and K2 == K and rast.cap >= K
    ys, xs = np.mgrid[0:cam.height, 0:cam.width]
    _compare_pixels(rast, 0, sc, cam, xs.reshape(-1).astype(np.int32), ys.reshape(-1).astype(np.int32))


# --------------------------------------------------------------------------
# step 4: gradients vs central finite differences of the FP64 oracle
# --------------------------------------------------------------------------

def _gpu_grads(P, n, M, cams, targets):
    rast, planes = gc.rasterize(P, n, M, cams)
    tgt = torch.from_numpy(np.concatenate([t.reshape(-1) for t in targets])).cuda()
    loss, dldc = rast.l1_loss(tgt)
    g = rast.backward(planes, dldc)
    torch.cuda.synchronize()
    return g.cpu().numpy().astype(np.float64), float(loss.sum().item()), rast


def _compare_blocks(g_gpu, g_fd, gp, gm, M, prims, label=""):
    checked = 0
    worst = 0.0
    for name, a, b in gc.groups(M):
        for col, i in enumerate(prims):
            fd = g_fd[a:b, col].copy()
            gg = g_gpu[a:b, i].copy()
            kink = np.abs(gp[a:b, col] - gm[a:b, col]) > 0.1 * np.maximum(np.abs(gp[a:b, col]), np.abs(gm[a:b, col])) + 1e-12
            fd[kink] = 0.0
            gg[kink] = 0.0
            nrm = np.linalg.norm(fd)
            if nrm <= gc.GRAD_MIN_NORM:
                continue
            rel = np.linalg.norm(gg - fd) / nrm
            worst = max(worst, rel)
            checked += 1
            assert rel <= gc.GRAD_RTOL, (label, name, i, rel, gg, fd)
    return checked, worst


def _tiny_scene(M, seed):
    rng = np.random.default_rng(seed)
    n = 24
    cam = scenes.pinhole(*scenes.look_at((0.0, 0.0, -3.0)), 48, 40)
    P = np.zeros((scenes.n_planes(M), 32), np.float32)
    P[6, :] = 1.0
    P[0:3, :n] = rng.uniform(-0.6, 0.6, (3, n))
    P[3:6, :n] = rng.normal(-2.6, 0.3, (3, n))
    P[6:10, :n] = rng.standard_normal((4, n))
    P[10, :n] = np.clip(rng.normal(0, 1.0, n), -3, 3)
    P[11, :n] = np.clip(rng.normal(0.2, 0.4, n), -1.0, 1.5)
    P[12:15, :n] = rng.uniform(0, 1, (3, n))
    for m in range(M):
        base = 15 + 6 * m
        # lobe axes within ~50 degrees of the view direction V = normalize(mu - campos)
        # (about +z here), so that R . V > 0 and every lobe term is active
        P[base, :n] = rng.uniform(0.15, 0.9, n)
        P[base + 1, :n] = rng.uniform(0, 2 * math.pi, n)
        P[base + 2, :n] = rng.normal(0, 0.3, n)
        P[base + 3:base + 6, :n] = rng.uniform(0, 0.5, (3, n))
    return P, n, cam


@pytest.mark.parametrize("M", [0, 1, 3])
def test_gradients_tiny_scene_all_parameters(M):
    P, n, cam = _tiny_scene(M, 40 + M)
    target = scenes.target_images([cam], seed=9)
    g_gpu, loss, _ = _gpu_grads(P, n, M, [cam], target)
    assert abs(loss - oracle.l1_loss(P, n, M, [cam], target)) < 1e-5
    g_fd, gp, gm = oracle.fd_grad(P, n, M, [cam], target, list(range(scenes.n_planes(M))), list(range(n)), local=False)
    checked, worst = _compare_blocks(g_gpu, g_fd, gp, gm, M, list(range(n)), f"M={M}")
    assert checked > n * 4


@pytest.mark.parametrize("kw", [dict(color_mode=1), dict(color_mode=2), dict(b_lo=0.0, b_hi=0.6),
                                dict(b_lo=-math.inf, b_hi=0.1, color_mode=2)])
def test_gradients_decomposition_modes(kw):
    """Sec. 4.3 decompositions, differentiated: diffuse-only (c = c0) and
    specular-only (c = lobes) colour and the geometry mask on b, each against
    central differences of the oracle rendered with the same option (tiny
    scene, every parameter of every primitive, 2 lobes).  Blocks the option
    zeroes (lobes under diffuse, c0 under specular, masked primitives) are
    checked to be zero on the GPU too."""
    M = 2
    P, n, cam = _tiny_scene(M, 60)
    target = scenes.target_images([cam], seed=10)
    gc.ensure_built()
    rast, planes = gc.rasterize(P, n, M, [cam], opts=_lib.default_opts(**kw))
    tgt = torch.from_numpy(target[0].reshape(-1)).cuda()
    loss, dldc = rast.l1_loss(tgt)
    g_gpu = rast.backward(planes, dldc).cpu().numpy().astype(np.float64)
    assert abs(float(loss.sum().item()) - oracle.l1_loss(P, n, M, [cam], target, **kw)) < 1e-5
    g_fd, gp, gm = oracle.fd_grad(P, n, M, [cam], target, list(range(scenes.n_planes(M))), list(range(n)),
                                  local=False, **kw)
    checked, _ = _compare_blocks(g_gpu, g_fd, gp, gm, M, list(range(n)), str(kw))
    assert checked >= n * 2      # the mask and the colour modes zero whole groups of blocks
    mode = kw.get("color_mode", 0)
    if mode == 1:
        assert np.all(g_gpu[15:15 + 6 * M, :n] == 0.0)
    if mode == 2:
        assert np.all(g_gpu[12:15, :n] == 0.0)
    if "b_lo" in kw:
        b = P[11, :n]
        masked = ~((b >= np.float32(kw["b_lo"])) & (b < np.float32(kw["b_hi"])))
        assert masked.any() and np.all(g_gpu[:, :n][:, masked] == 0.0)


@pytest.mark.parametrize("cfg,nblocks", [(2, 24), (3, 12)])
def test_gradients_sampled_blocks_full_size(cfg, nblocks):
    """Full-size workloads: gradients of sampled primitives (every parameter)
    against finite differences over the sub-scene that can touch their pixels."""
    sc = scenes.config_scene(cfg)
    cam = sc.cameras[0]
    target = scenes.target_images([cam], seed=17)
    g_gpu, _, rast = _gpu_grads(sc.planes, sc.n, sc.n_lobes, [cam], target)
    _, rects, keys = gc.proj_arrays(rast)
    rng = np.random.default_rng(cfg)
    vis = np.nonzero(keys[0, :sc.n] != 0xFFFFFFFF)[0]
    chosen = rng.choice(vis, size=nblocks, replace=False)
    pr_all = oracle.project(sc.planes, sc.n, sc.n_lobes, cam)
    total = 0
    for i in chosen:
        a, _, c = pr_all["cov"][i]
        mx, my = pr_all["mu2"][i]
        ex, ey = math.sqrt(a) + 3, math.sqrt(c) + 3
        x0, x1 = max(0, int(mx - ex)), min(cam.width - 1, int(mx + ex) + 1)
        y0, y1 = max(0, int(my - ey)), min(cam.height - 1, int(my + ey) + 1)
        idx = gc.sub_scene(sc.planes, sc.n, sc.n_lobes, cam, x0, x1, y0, y1, pr=pr_all)
        sub = np.ascontiguousarray(sc.planes[:, idx])
        j = int(np.nonzero(idx == i)[0][0])
        g_fd, gp, gm = oracle.fd_grad(sub, len(idx), sc.n_lobes, [cam], target,
                                      list(range(scenes.n_planes(sc.n_lobes))), [j], local=True)
        checked, _ = _compare_blocks(g_gpu[:, [i]], g_fd, gp, gm, sc.n_lobes, [0], f"cfg{cfg} prim {i}")
        total += checked
    assert total >= nblocks


def test_autograd_function_matches_direct_backward():
    sc = scenes.config_scene(1, n=1024)
    cam = scenes.pinhole(*scenes.look_at((0.0, 0.0, -3.0)), 64, 48)
    gc.ensure_built()
    planes = torch.from_numpy(sc.planes).cuda().requires_grad_(True)
    rast = render.Rasterizer(sc.n, sc.pitch, sc.n_lobes, [cam])
    tgt = torch.from_numpy(scenes.target_images([cam], seed=3)[0].reshape(-1)).cuda()
    color = render.render(planes, rast)
    loss = (color - tgt).abs().mean()
    loss.backward()
    loss2, dldc = rast.l1_loss(tgt)
    assert abs(float(loss2.item()) - float(loss.item())) < 1e-6
    g2 = rast.backward(planes.detach(), dldc)
    torch.cuda.synchronize()
    assert torch.allclose(planes.grad, g2, rtol=1e-5, atol=1e-9)


def test_l1_kernel_matches_numpy():
    cams = [scenes.pinhole(*scenes.look_at((0.0, 0.0, -3.0)), w, h) for (w, h) in ((33, 17), (64, 64))]
    gc.ensure_built()
    rast = render.Rasterizer(1, 32, 0, cams)
    rng = np.random.default_rng(0)
    col = rng.uniform(0, 1, 3 * rast.total_pixels).astype(np.float32)
    tgt = rng.uniform(0, 1, 3 * rast.total_pixels).astype(np.float32)
    tgt[5] = col[5]
    rast.color.copy_(torch.from_numpy(col))
    loss, d = rast.l1_loss(torch.from_numpy(tgt).cuda())
    loss, d = loss.cpu().numpy(), d.cpu().numpy()
    off = 0
    for v, c in enumerate(cams):
        hw = c.width * c.height
        seg = slice(3 * off, 3 * off + 3 * hw)
        diff = col[seg].astype(np.float64) - tgt[seg]
        assert abs(loss[v] - np.abs(diff).mean()) < 1e-6
        assert np.allclose(d[seg], np.sign(diff) / (3 * hw), rtol=1e-6, atol=0)
        off += hw
    assert d[5] == 0.0


@pytest.mark.parametrize("tile,persistent", [((16, 8), False), ((16, 16), False), ((16, 8), True)])
def test_forward_with_fused_l1_equals_separate_calls(tile, persistent):
    """beta_raster_fwd_l1 = beta_raster_fwd then beta_l1_loss (one CTA per
    tile, or the persistent longest-first schedule): the image, T and
    n_contrib bit for bit, dL/dC bit for bit (the same sign of the same fp32
    difference), the per-view loss to fp32 summation order."""
    sc = scenes.config_scene(4, n=40_000, n_views=8)
    cams = sc.cameras[::2]                                  # four sizes, ragged edge tiles
    opts = _lib.default_opts(tile_w=tile[0], tile_h=tile[1])
    gc.ensure_built()
    planes = torch.from_numpy(np.ascontiguousarray(sc.planes)).cuda()
    rast = render.Rasterizer(sc.n, sc.pitch, sc.n_lobes, cams, opts, persistent=persistent)
    rast.forward(planes)
    torch.cuda.synchronize()
    tgt_np = np.concatenate([t.reshape(-1) for t in scenes.target_images(cams, seed=3)])
    target = torch.from_numpy(tgt_np).cuda()
    rast.raster_fwd(planes)
    loss_a, d_a = (x.clone() for x in rast.l1_loss(target))
    img_a, T_a, n_a = rast.color.clone(), rast.T_final.clone(), rast.n_contrib.clone()
    rast.color.zero_(); rast.T_final.zero_(); rast.dL_dcolor.zero_(); rast.loss.zero_()
    if persistent:
        rast.schedule()
    loss_b, d_b = rast.raster_fwd_l1(planes, target)
    torch.cuda.synchronize()
    assert torch.equal(rast.color, img_a) and torch.equal(rast.T_final, T_a)
    assert torch.equal(rast.n_contrib, n_a)
    assert torch.equal(d_b, d_a)
    la, lb = loss_a.cpu().numpy().astype(np.float64), loss_b.cpu().numpy().astype(np.float64)
    assert np.all(la > 0) and np.max(np.abs(la - lb) / la) < 1e-5


@pytest.mark.parametrize("tile,bs,persistent", [((16, 8), 64, False), ((16, 8), 128, True), ((8, 8), 64, False),
                                                ((16, 16), 256, True), ((32, 16), 128, False)])
def test_forward_backward_in_one_launch_equals_separate_calls(tile, bs, persistent):
    """beta_raster_fwd_bwd_l1 = beta_raster_fwd_l1 then beta_raster_bwd of
    its dL/dC: image, T, n_contrib and dL/dC bit for bit, the per-view loss
    bit for bit (the same tile partials summed in the same order), and the
    2D-gradient sums within 1e-5 of each field's largest value (the same
    terms, added by atomics in another order).  Without the optional state
    buffers the image, loss and gradients are the same.  8x4 tiles, which
    have no pixel-pair kernels, are refused."""
    sc = scenes.config_scene(4, n=40_000, n_views=8)
    cams = sc.cameras[::2]                                  # four sizes, ragged edge tiles
    opts = _lib.default_opts(tile_w=tile[0], tile_h=tile[1], batch_s=bs)
    gc.ensure_built()
    planes = torch.from_numpy(np.ascontiguousarray(sc.planes)).cuda()
    target = torch.from_numpy(np.concatenate([t.reshape(-1) for t in scenes.target_images(cams, seed=7)])).cuda()
    rast = render.Rasterizer(sc.n, sc.pitch, sc.n_lobes, cams, opts, persistent=persistent)
    rast.forward(planes)
    if persistent:
        rast.schedule()
    loss_a, d_a = (x.clone() for x in rast.raster_fwd_l1(planes, target))
    img_a, T_a, n_a = rast.color.clone(), rast.T_final.clone(), rast.n_contrib.clone()
    rast.raster_bwd(planes, rast.dL_dcolor)
    g2_a = rast.grad2d.clone()
    rast.grad2d.zero_()
    out = []
    for keep in (True, False):
        rast.color.zero_(); rast.T_final.zero_(); rast.n_contrib.zero_(); rast.dL_dcolor.zero_()
        rast.loss.zero_(); rast.grad2d.zero_()
        if persistent:
            rast.schedule()
        rast.raster_fwd_bwd_l1(planes, target, keep_state=keep)
        torch.cuda.synchronize()
        out.append((rast.color.clone(), rast.loss.clone(), rast.grad2d.clone(), rast.T_final.clone(),
                    rast.n_contrib.clone(), rast.dL_dcolor.clone()))
    g_ref = g2_a.view(-1, 12)[:, :10].cpu().numpy().astype(np.float64)
    scale = np.abs(g_ref).max(axis=0) + 1e-30
    assert np.all(np.abs(g_ref).max(axis=0) > 0)
    for k, (img, loss, g2, T, nc, d) in enumerate(out):
        assert torch.equal(img, img_a) and torch.equal(loss, loss_a)
        g = g2.view(-1, 12)[:, :10].cpu().numpy().astype(np.float64)
        assert np.max(np.abs(g - g_ref) / scale) < 1e-5
        assert bool((g2.view(-1, 12)[:, 10:] == 0).all())
        if k == 0:
            assert torch.equal(T, T_a) and torch.equal(nc, n_a) and torch.equal(d, d_a)
        else:                                               # not written without their buffers
            assert bool((T == 0).all()) and bool((nc == 0).all()) and bool((d == 0).all())
    r84 = render.Rasterizer(sc.n, sc.pitch, sc.n_lobes, cams, _lib.default_opts(tile_w=8, tile_h=4))
    assert not r84.fused_supported
    with pytest.raises(_lib.BetaError) as e:
        r84.raster_fwd_bwd_l1(planes, target)
    assert e.value.code == _lib.BETA_ERR_ARG
