"""Shared helpers of the GPU parity tests (CUDA path vs FP64 oracle)."""
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


def proj_arrays(rast):
    """(records (V,pitch,12) f32, rects (V,pitch,4) int, keys (V,pitch) u32) from the proj buffer."""
    V, pitch = rast.V, rast.pitch
    raw = rast.proj.cpu().numpy()
    nrec = V * pitch
    rec = raw[:nrec * 48].view(np.float32).reshape(V, pitch, 12)
    rr = raw[nrec * 48:nrec * 56].view(np.uint32).reshape(V, pitch, 2)
    rects = np.stack([rr[..., 0] & 0xFFFF, rr[..., 0] >> 16, rr[..., 1] & 0xFFFF, rr[..., 1] >> 16], -1).astype(np.int64)
    keys = raw[nrec * 56:nrec * 60].view(np.uint32).reshape(V, pitch)
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
    """Primitive id of each pixel's last contributor (-1 if none)."""
    cam = rast.cameras[v]
    nc = rast.plane(rast.n_contrib, v).cpu().numpy().astype(np.int64)
    ranges = rast.ranges.cpu().numpy().view(np.uint32).astype(np.int64)
    K = int(rast.count.item())
    vals = rast.pair_vals[:max(K, 1)].cpu().numpy().view(np.uint32).astype(np.int64)
    ntx = (cam.width + 15) // 16
    toff = 0
    for u in range(v):
        c = rast.cameras[u]
        toff += ((c.width + 15) // 16) * ((c.height + 15) // 16)
    ys, xs = np.mgrid[0:cam.height, 0:cam.width]
    g = toff + (ys // 16) * ntx + (xs // 16)
    pos = ranges[g] + nc - 1
    out = np.where(nc > 0, vals[np.clip(pos, 0, max(K - 1, 0))] - v * pitch, -1)
    return out


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
