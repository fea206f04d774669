"""Shared helpers of the GPU parity tests (CUDA path vs FP64 oracle)."""
import math

import numpy as np
import torch

import oracle
from paper_2501_18630_gb300 import _lib, build, render, scenes

IMG_TOL = 2e-5      # absolute per channel (FP32 image vs FP64 oracle)
GRAD_RTOL = 1e-3    # relative, per (primitive, parameter group) block
GRAD_MIN_NORM = 1e-6

GROUPS = [("mean", 0, 3), ("log_scale", 3, 6), ("quat", 6, 10), ("opacity", 10, 11), ("b", 11, 12),
          ("c0", 12, 15)]


def groups(n_lobes):
    g = list(GROUPS)
    for m in range(n_lobes):
        b = 15 + 6 * m
        g += [(f"lobe{m}_dir", b, b + 2), (f"lobe{m}_b", b + 2, b + 3), (f"lobe{m}_c", b + 3, b + 6)]
    return g


_built = False


def ensure_built():
    global _built
    if not _built:
        build.build()
        oracle.build()
        _built = True


def rasterize(planes_np, n, n_lobes, cams, opts=None, cap=None, check=True):
    ensure_built()
    planes = torch.from_numpy(np.ascontiguousarray(planes_np)).cuda()
    rast = render.Rasterizer(n, planes_np.shape[1], n_lobes, cams, opts, pair_capacity=cap)
    rast.forward(planes, check_capacity=check)
    torch.cuda.synchronize()
    return rast, planes


def proj_arrays(rast, with_tiles=False):
    """(records (V,pitch,12) f32, rects (V,pitch,4) int, keys (V,pitch) u32[, rule B2 tile
    masks (V,pitch) u32]) from the proj buffer."""
    V, pitch = rast.V, rast.pitch
    raw = rast.proj.cpu().numpy()
    nrec = V * pitch
    rec = raw[:nrec * 48].view(np.float32).reshape(V, pitch, 12)
    rr = raw[nrec * 48:nrec * 56].view(np.uint32).reshape(V, pitch, 2)
    rects = np.stack([rr[..., 0] & 0xFFFF, rr[..., 0] >> 16, rr[..., 1] & 0xFFFF, rr[..., 1] >> 16], -1).astype(np.int64)
    keys = raw[nrec * 56:nrec * 60].view(np.uint32).reshape(V, pitch)
    if with_tiles:
        return rec, rects, keys, raw[nrec * 60:nrec * 64].view(np.uint32).reshape(V, pitch)
    return rec, rects, keys


def sorted_pairs(rast):
    st, K = rast.device_status()
    assert st == 0, st
    ranges = rast.ranges.cpu().numpy().view(np.uint32)
    vals = rast.pair_vals[:K].cpu().numpy().view(np.uint32)
    return K, ranges, vals


def image(rast, v):
    return rast.image(rast.color, v).cpu().numpy().astype(np.float64)


def last_ids(rast, v, pitch):
    """Primitive id of each pixel's last contributor (-1 if none), from
    n_contrib (1 + position in the pixel's tile list) under the rasterizer's
    own tile shape."""
    cam = rast.cameras[v]
    tw, th = int(rast.opts.tile_w), int(rast.opts.tile_h)
    nc = rast.plane(rast.n_contrib, v).cpu().numpy().astype(np.int64)
    ranges = rast.ranges.cpu().numpy().view(np.uint32).astype(np.int64)
    K = int(rast.count.item())
    vals = rast.pair_vals[:max(K, 1)].cpu().numpy().view(np.uint32).astype(np.int64)
    ntx = (cam.width + tw - 1) // tw
    toff = 0
    for u in range(v):
        c = rast.cameras[u]
        toff += ((c.width + tw - 1) // tw) * ((c.height + th - 1) // th)
    ys, xs = np.mgrid[0:cam.height, 0:cam.width]
    g = toff + (ys // th) * ntx + (xs // tw)
    pos = ranges[g] + nc - 1
    assert np.all((nc == 0) | (nc <= ranges[g + 1] - ranges[g])), "n_contrib beyond its tile list"
    out = np.where(nc > 0, vals[np.clip(pos, 0, max(K - 1, 0))] - v * pitch, -1)
    return out


def r2_fp64(pr, ids, xs, ys):
    """FP64 r^2 of primitives ids[k] at pixel centres (xs[k], ys[k]) (Eq. r)."""
    ids = np.asarray(ids)
    dx = xs + 0.5 - pr["mu2"][ids, 0]
    dy = ys + 0.5 - pr["mu2"][ids, 1]
    A, B, C = pr["conic"][ids, 0], pr["conic"][ids, 1], pr["conic"][ids, 2]
    return A * dx * dx + 2.0 * B * dx * dy + C * dy * dy


def unexplained_last_mismatches(last_gpu, last_or, T_or, xs, ys, pr, t_eps=2.0 ** -19, band=1e-4):
    """Pixels whose last contributor differs between the CUDA path and the
    FP64 oracle for a reason other than the two that make it legitimately
    differ: a support-boundary decision (the later of the two primitives has
    FP64 r^2 within `band` of 1, where its alpha is below o * band^beta) or
    an early-termination decision (the oracle's final T within 1e-3 of
    t_eps).  Returns the indices of the unexplained pixels."""
    mism = np.nonzero(last_gpu != last_or)[0]
    bad = []
    for k in mism:
        cand = [int(i) for i in (last_gpu[k], last_or[k]) if i >= 0]
        r2 = r2_fp64(pr, cand, np.full(len(cand), xs[k]), np.full(len(cand), ys[k]))
        near_edge = np.any(np.abs(r2 - 1.0) < band)
        near_stop = abs(T_or[k] - t_eps) < 1e-3 * t_eps or T_or[k] < t_eps
        if not (near_edge or near_stop):
            bad.append(k)
    return np.asarray(bad, np.int64), len(mism)


def fd_block_views(planes, n, n_lobes, cams, targets, i, prs=None, margin=3.0):
    """Central finite differences (and one-sided estimates) of sum_v L1_v
    w.r.t. every raw parameter of primitive i, each view evaluated on the
    sub-scene that can touch the primitive's padded support box there.
    Returns (g, gp, gm) of shape (n_planes, 1)."""
    P = planes.shape[0]
    g = np.zeros((P, 1)); gp = np.zeros((P, 1)); gm = np.zeros((P, 1))
    for v, cam in enumerate(cams):
        pr = prs[v] if prs is not None else oracle.project(planes, n, n_lobes, cam)
        if not pr["valid"][i]:
            continue
        a, _, c = pr["cov"][i]
        mx, my = pr["mu2"][i]
        ex, ey = math.sqrt(a) + margin, math.sqrt(c) + margin
        x0, x1 = max(0, int(mx - ex)), min(cam.width - 1, int(mx + ex) + 1)
        y0, y1 = max(0, int(my - ey)), min(cam.height - 1, int(my + ey) + 1)
        if x0 > x1 or y0 > y1:
            continue
        idx = sub_scene(planes, n, n_lobes, cam, x0, x1, y0, y1, pr=pr)
        sub = np.ascontiguousarray(planes[:, idx])
        j = int(np.nonzero(idx == i)[0][0])
        a_, b_, c_ = oracle.fd_grad(sub, len(idx), n_lobes, [cam], [targets[v]], list(range(P)), [j],
                                    local=True)
        g += a_; gp += b_; gm += c_
    return g, gp, gm


def sub_scene(planes, n, n_lobes, cam, x0, x1, y0, y1, margin=2.0, pr=None):
    """Primitives whose FP64 support box meets the pixel box [x0,x1]x[y0,y1]
    (all others have r^2 >= 1 there, so the pixels render identically)."""
    pr = pr if pr is not None else oracle.project(planes, n, n_lobes, cam)
    a, c = pr["cov"][:, 0], pr["cov"][:, 2]
    mx, my = pr["mu2"][:, 0], pr["mu2"][:, 1]
    ex, ey = np.sqrt(np.maximum(a, 0)) + margin, np.sqrt(np.maximum(c, 0)) + margin
    keep = (pr["valid"] > 0) & (mx + ex >= x0) & (mx - ex <= x1 + 1) & (my + ey >= y0) & (my - ey <= y1 + 1)
    idx = np.nonzero(keep)[0]
    return idx
