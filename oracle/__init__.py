"""FP64 CPU oracle of the Beta-splatting rasterizer (test infrastructure).

Only tests/, __graft_entry__.smoke() and bench.py's cpu_baseline and
reference legs may import this package.  The product path never does: it
runs on the CUDA library and fails loudly without it.

The arithmetic lives in beta_oracle.c (plain FP64 C, one pixel at a time over
every primitive, Sec. 3.2 / Eq. C of arXiv 2501.18630).  This module compiles
it with gcc, marshals arguments, and adds three pieces written on top of it:

  * bin_pairs(): the sorted (tile, primitive) list implied by rule B1 and
    rule D, by expanding rectangles and calling numpy's lexsort;
  * loss_and_fd_grad(): central finite differences of the FP64 L1 loss;
  * render_full(): a whole image, for small workloads.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import sys
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "beta_oracle.c")
_LIB_PATH = os.path.join(_HERE, "_beta_oracle.so")
_lock = threading.Lock()
_lib = None

DEFAULT_T_EPS = 2.0 ** -19
DEFAULT_ALPHA_MAX = 0.99


def build(force: bool = False) -> str:
    """Compile beta_oracle.c into _beta_oracle.so (gcc, no FMA contraction)."""
    if not force and os.path.exists(_LIB_PATH) and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
           "-D_GNU_SOURCE", _SRC, "-o", tmp, "-lm", "-lpthread"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class OCam(ctypes.Structure):
    _fields_ = [("R", ctypes.c_double * 9), ("t", ctypes.c_double * 3),
                ("fx", ctypes.c_double), ("fy", ctypes.c_double), ("cx", ctypes.c_double),
                ("cy", ctypes.c_double), ("near_plane", ctypes.c_double),
                ("width", ctypes.c_int32), ("height", ctypes.c_int32), ("bg", ctypes.c_double * 3)]


class OOpts(ctypes.Structure):
    _fields_ = [("t_eps", ctypes.c_double), ("alpha_max", ctypes.c_double),
                ("blur_eps", ctypes.c_double), ("color_mode", ctypes.c_int32),
                ("n_threads", ctypes.c_int32), ("b_lo", ctypes.c_double), ("b_hi", ctypes.c_double)]


class OPrim(ctypes.Structure):
    _fields_ = [("valid", ctypes.c_int32), ("key", ctypes.c_uint32), ("depth", ctypes.c_double),
                ("mu2", ctypes.c_double * 2), ("cov", ctypes.c_double * 3),
                ("conic", ctypes.c_double * 3), ("o", ctypes.c_double), ("beta", ctypes.c_double),
                ("color", ctypes.c_double * 3)]


def lib():
    global _lib
    with _lock:
        if _lib is None:
            path = build()
            L = ctypes.CDLL(path)
            dp, ip, up, fp = (ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int32),
                              ctypes.POINTER(ctypes.c_uint32), ctypes.POINTER(ctypes.c_float))
            L.oracle_render.restype = ctypes.c_int32
            L.oracle_render.argtypes = [dp, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                        ctypes.POINTER(OCam), ctypes.POINTER(OOpts), ip, ip,
                                        ctypes.c_int32, dp, dp, ip, ip]
            L.oracle_project.restype = None
            L.oracle_project.argtypes = [dp, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                         ctypes.POINTER(OCam), ctypes.POINTER(OOpts), ctypes.POINTER(OPrim)]
            L.oracle_rule_exp.restype = ctypes.c_float
            L.oracle_rule_exp.argtypes = [ctypes.c_float]
            L.oracle_rule_opacity.restype = None
            L.oracle_rule_opacity.argtypes = [fp, ctypes.c_int32, fp]
            L.oracle_rule_rects.restype = None
            L.oracle_rule_rects.argtypes = [fp, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                            ctypes.POINTER(OCam), ctypes.c_float, ctypes.c_float,
                                            ctypes.c_float, ctypes.c_int32, ctypes.c_int32, ip, up, ip, up]
            _lib = L
    return _lib


def _ptr(a, ctype):
    return a.ctypes.data_as(ctypes.POINTER(ctype))


def make_cam(cam) -> OCam:
    """scenes.Camera -> OCam (fp32 values widened exactly to fp64)."""
    c = OCam()
    R = np.asarray(cam.R, np.float32).astype(np.float64).reshape(-1)
    t = np.asarray(cam.t, np.float32).astype(np.float64)
    for k in range(9):
        c.R[k] = R[k]
    for k in range(3):
        c.t[k] = t[k]
        c.bg[k] = float(np.float32(cam.bg[k]))
    c.fx, c.fy = float(np.float32(cam.fx)), float(np.float32(cam.fy))
    c.cx, c.cy = float(np.float32(cam.cx)), float(np.float32(cam.cy))
    c.near_plane = float(np.float32(cam.near))
    c.width, c.height = int(cam.width), int(cam.height)
    return c


def make_opts(t_eps=DEFAULT_T_EPS, alpha_max=DEFAULT_ALPHA_MAX, blur_eps=0.0, color_mode=0,
              n_threads=None, b_lo=-np.inf, b_hi=np.inf) -> OOpts:
    o = OOpts()
    o.b_lo = float(np.float32(b_lo))
    o.b_hi = float(np.float32(b_hi))
    o.t_eps = float(np.float32(t_eps))
    o.alpha_max = float(np.float32(alpha_max))
    o.blur_eps = float(np.float32(blur_eps))
    o.color_mode = int(color_mode)
    o.n_threads = int(n_threads or os.cpu_count() or 1)
    return o


def _planes64(planes):
    return np.ascontiguousarray(planes, dtype=np.float64)


def render(planes, n, n_lobes, cam, xs, ys, **opts):
    """FP64 colour (npix,3), transmittance (npix,), last contributor id (npix,),
    contributor count (npix,) at the integer pixels (xs[k], ys[k])."""
    L = lib()
    p = _planes64(planes)
    xs = np.ascontiguousarray(xs, np.int32)
    ys = np.ascontiguousarray(ys, np.int32)
    npix = xs.shape[0]
    C = np.zeros((npix, 3), np.float64)
    T = np.zeros(npix, np.float64)
    last = np.zeros(npix, np.int32)
    cnt = np.zeros(npix, np.int32)
    oc, oo = make_cam(cam), make_opts(**opts)
    L.oracle_render(_ptr(p, ctypes.c_double), n, p.shape[1], n_lobes, ctypes.byref(oc),
                    ctypes.byref(oo), _ptr(xs, ctypes.c_int32), _ptr(ys, ctypes.c_int32), npix,
                    _ptr(C, ctypes.c_double), _ptr(T, ctypes.c_double), _ptr(last, ctypes.c_int32),
                    _ptr(cnt, ctypes.c_int32))
    return C, T, last, cnt


def render_full(planes, n, n_lobes, cam, **opts):
    """Whole image: colour (3,H,W), T (H,W), last (H,W), count (H,W)."""
    W, H = cam.width, cam.height
    ys, xs = np.meshgrid(np.arange(H, dtype=np.int32), np.arange(W, dtype=np.int32), indexing="ij")
    C, T, last, cnt = render(planes, n, n_lobes, cam, xs.reshape(-1), ys.reshape(-1), **opts)
    return (C.reshape(H, W, 3).transpose(2, 0, 1), T.reshape(H, W), last.reshape(H, W),
            cnt.reshape(H, W))


def project(planes, n, n_lobes, cam, **opts):
    """Per-primitive FP64 quantities as a dict of numpy arrays."""
    L = lib()
    p = _planes64(planes)
    out = (OPrim * max(n, 1))()
    oc, oo = make_cam(cam), make_opts(**opts)
    L.oracle_project(_ptr(p, ctypes.c_double), n, p.shape[1], n_lobes, ctypes.byref(oc),
                     ctypes.byref(oo), out)
    raw = np.ctypeslib.as_array(ctypes.cast(out, ctypes.POINTER(ctypes.c_uint8)),
                                shape=(max(n, 1) * ctypes.sizeof(OPrim),)).copy()
    dt = np.dtype([("valid", np.int32), ("key", np.uint32), ("depth", np.float64),
                   ("mu2", np.float64, 2), ("cov", np.float64, 3), ("conic", np.float64, 3),
                   ("o", np.float64), ("beta", np.float64), ("color", np.float64, 3)])
    assert dt.itemsize == ctypes.sizeof(OPrim)
    rec = raw.view(dt)[:n]
    return {k: np.array(rec[k]) for k in dt.names}


def rule_exp(x: float) -> float:
    return float(lib().oracle_rule_exp(ctypes.c_float(x)))


def rule_opacity(logit) -> np.ndarray:
    """The fixed fp32 opacity rule of the relocation step (float32 array)."""
    x = np.ascontiguousarray(np.asarray(logit, np.float32))
    out = np.empty_like(x)
    fp = ctypes.POINTER(ctypes.c_float)
    lib().oracle_rule_opacity(x.ctypes.data_as(fp), int(x.size), out.ctypes.data_as(fp))
    return out


def rule_rects(planes, n, n_lobes, cam, blur_eps=0.0, tile_w=16, tile_h=16, b_lo=-np.inf, b_hi=np.inf,
               with_tiles=False):
    """Rule B1 rectangles (n,4) = (tx0, tx1, ty0, ty1), rule D keys (n,), binned flags (n,),
    and with with_tiles the rule B2 tile masks (n,) of the rectangles (bit r w + q for tile
    (tx0 + q, ty0 + r); 0xFFFFFFFF for rectangles of more than 32 tiles: every tile).
    Primitives with b outside [b_lo, b_hi) are not binned (geometry decomposition)."""
    L = lib()
    p = np.ascontiguousarray(planes, dtype=np.float32)
    rects = np.zeros((max(n, 1), 4), np.int32)
    keys = np.zeros(max(n, 1), np.uint32)
    binned = np.zeros(max(n, 1), np.int32)
    tiles = np.zeros(max(n, 1), np.uint32)
    oc = make_cam(cam)
    L.oracle_rule_rects(_ptr(p, ctypes.c_float), n, p.shape[1], n_lobes, ctypes.byref(oc),
                        ctypes.c_float(np.float32(blur_eps)), ctypes.c_float(np.float32(b_lo)),
                        ctypes.c_float(np.float32(b_hi)), tile_w, tile_h,
                        _ptr(rects, ctypes.c_int32), _ptr(keys, ctypes.c_uint32),
                        _ptr(binned, ctypes.c_int32), _ptr(tiles, ctypes.c_uint32))
    if with_tiles:
        return rects[:n], keys[:n], binned[:n], tiles[:n]
    return rects[:n], keys[:n], binned[:n]


def expand_tiles(rects, tiles):
    """(primitive row, tx, ty) of every tile a primitive's rule B2 mask keeps
    inside its rectangle, in rectangle row-major order."""
    r = rects.astype(np.int64)
    w = r[:, 1] - r[:, 0] + 1
    h = r[:, 3] - r[:, 2] + 1
    cnt = w * h
    rw = np.repeat(np.arange(len(r)), cnt)
    local = np.arange(cnt.sum(), dtype=np.int64) - np.repeat(np.cumsum(cnt) - cnt, cnt)
    full = np.repeat(cnt > 32, cnt)
    bit = (tiles.astype(np.uint64)[rw] >> np.minimum(local, 31).astype(np.uint64)) & np.uint64(1)
    keep = full | (bit == 1)
    rw, local = rw[keep], local[keep]
    ty = r[rw, 2] + local // w[rw]
    tx = r[rw, 0] + local % w[rw]
    return rw, tx, ty


def n_tiles(cam, tile_w=16, tile_h=16):
    return (cam.width + tile_w - 1) // tile_w, (cam.height + tile_h - 1) // tile_h


def bin_pairs(planes, n, n_lobes, cams, blur_eps=0.0, tile_w=16, tile_h=16, pitch=None,
              b_lo=-np.inf, b_hi=np.inf):
    """Sorted (global tile, record) pairs of a batch of views: one pair per
    tile of a primitive's rule B1 rectangle that its rule B2 mask keeps.

    A record is view * pitch + primitive.  Global tiles are numbered view by
    view, row-major inside a view.  The order is (tile, depth key, primitive
    index) ascending.  Returns (tiles uint32[K], records uint32[K],
    ranges uint32[T_total + 1]).
    """
    pitch = pitch or planes.shape[1]
    all_tiles, all_keys, all_rec = [], [], []
    tile_off = 0
    for v, cam in enumerate(cams):
        rects, keys, binned, masks = rule_rects(planes, n, n_lobes, cam, blur_eps, tile_w, tile_h, b_lo, b_hi,
                                                with_tiles=True)
        ntx, nty = n_tiles(cam, tile_w, tile_h)
        idx = np.nonzero(binned)[0]
        rw, tx, ty = expand_tiles(rects[idx], masks[idx])
        prim = idx[rw]
        all_tiles.append(tile_off + ty * ntx + tx)
        all_keys.append(keys[prim].astype(np.int64))
        all_rec.append(v * pitch + prim.astype(np.int64))
        tile_off += ntx * nty
    tiles = np.concatenate(all_tiles) if all_tiles else np.zeros(0, np.int64)
    keys = np.concatenate(all_keys) if all_keys else np.zeros(0, np.int64)
    recs = np.concatenate(all_rec) if all_rec else np.zeros(0, np.int64)
    order = np.lexsort((recs, keys, tiles))
    tiles, recs = tiles[order], recs[order]
    ranges = np.searchsorted(tiles, np.arange(tile_off + 1), side="left").astype(np.uint32)
    return tiles.astype(np.uint32), recs.astype(np.uint32), ranges


def l1_loss(planes, n, n_lobes, cams, targets, pixel_sets=None, **opts):
    """Sum over views of mean |C - target| over 3HW (FP64).  With pixel_sets,
    only the listed pixels are summed (still divided by 3HW)."""
    total = 0.0
    for v, cam in enumerate(cams):
        if pixel_sets is None:
            C, _, _, _ = render_full(planes, n, n_lobes, cam, **opts)
            total += np.abs(C - targets[v].astype(np.float64)).sum() / (3.0 * cam.width * cam.height)
        else:
            xs, ys = pixel_sets[v]
            if len(xs) == 0:
                continue
            C, _, _, _ = render(planes, n, n_lobes, cam, xs, ys, **opts)
            tg = targets[v].astype(np.float64)[:, ys, xs].T
            total += np.abs(C - tg).sum() / (3.0 * cam.width * cam.height)
    return total


def support_pixels(planes, n, n_lobes, cam, i, margin=2.0, **opts):
    """Pixels whose centre lies inside the padded bounding box of primitive i's
    FP64 support ellipse (every pixel the primitive can touch)."""
    pr = project(planes[:, :], n, n_lobes, cam, **{k: v for k, v in opts.items()
                                                   if k in ("blur_eps", "color_mode", "b_lo", "b_hi")})
    if not pr["valid"][i]:
        return np.zeros(0, np.int32), np.zeros(0, np.int32)
    a, _, c = pr["cov"][i]
    mx, my = pr["mu2"][i]
    ex, ey = np.sqrt(a) + margin, np.sqrt(c) + margin
    x0, x1 = max(0, int(np.floor(mx - ex))), min(cam.width - 1, int(np.ceil(mx + ex)))
    y0, y1 = max(0, int(np.floor(my - ey))), min(cam.height - 1, int(np.ceil(my + ey)))
    if x0 > x1 or y0 > y1:
        return np.zeros(0, np.int32), np.zeros(0, np.int32)
    ys, xs = np.meshgrid(np.arange(y0, y1 + 1, dtype=np.int32), np.arange(x0, x1 + 1, dtype=np.int32), indexing="ij")
    return xs.reshape(-1), ys.reshape(-1)


def fd_grad(planes, n, n_lobes, cams, targets, plane_ids, prim_ids, rel_step=1e-6, local=True, **opts):
    """Central finite differences of the FP64 L1 loss w.r.t. planes[j, i] for
    every j in plane_ids and i in prim_ids.  Returns (len(plane_ids),
    len(prim_ids)) central estimates and the two one-sided estimates (for
    kink detection).  With local=True only pixels in the perturbed primitive's
    padded support box are re-rendered (the rest of the loss cancels)."""
    base = np.array(planes, dtype=np.float64, copy=True)
    g = np.zeros((len(plane_ids), len(prim_ids)))
    gp = np.zeros_like(g)
    gm = np.zeros_like(g)
    for b, i in enumerate(prim_ids):
        pix = None
        if local:
            pix = []
            for cam in cams:
                # union of the support boxes before and after a generous perturbation
                pix.append(support_pixels(base, n, n_lobes, cam, i, margin=3.0, **opts))
        f0 = l1_loss(base, n, n_lobes, cams, targets, pix, **opts)
        for a, j in enumerate(plane_ids):
            x0 = base[j, i]
            h = rel_step * max(1.0, abs(x0))
            base[j, i] = x0 + h
            fp = l1_loss(base, n, n_lobes, cams, targets, pix, **opts)
            base[j, i] = x0 - h
            fm = l1_loss(base, n, n_lobes, cams, targets, pix, **opts)
            base[j, i] = x0
            g[a, b] = (fp - fm) / (2.0 * h)
            gp[a, b] = (fp - f0) / h
            gm[a, b] = (f0 - fm) / h
    return g, gp, gm
