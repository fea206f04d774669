"""Seeded synthetic scenes and cameras for the Beta rasterizer.

This module only draws random numbers and builds camera poses.  It holds
none of the rasterizer's arithmetic, so both the CUDA path and the FP64
oracle can take their inputs from it.

Parameter layout (one float32 plane per scalar, planes of length `pitch`):

    0-2   mean x, y, z                      (mu, Sec. 3.2)
    3-5   log-scale (s = exp(.))            (s, Sec. 3.2)
    6-9   quaternion w, x, y, z (raw)        (q, Sec. 3.2)
    10    opacity logit (o = sigmoid(.))     (o, Sec. 3.2)
    11    Beta shape b (beta = 4 e^b)        (b, Eq. eq:beta)
    12-14 base colour c0 r, g, b             (c0, Sec. 3.3)
    15+6m lobe m: theta, phi, b_m, c_m r, g, b  (Sec. 3.3, 3+6M features)

so a primitive with M lobes carries 15 + 6M floats.

Cameras follow the OpenCV convention: x right, y down, z forward; a world
point X maps to camera space as R @ X + t.  The principal point is the
image centre and fx = fy = (W/2) / tan(fov_x/2).
"""
from __future__ import annotations

import dataclasses
import hashlib
import math

import numpy as np

SEED_BASE = 20250130

P_MEAN, P_LOGSCALE, P_QUAT, P_OPACITY, P_B, P_C0, P_LOBES = 0, 3, 6, 10, 11, 12, 15
LOBE_STRIDE = 6


def n_planes(n_lobes: int) -> int:
    """Floats per primitive: 15 geometry/base-colour scalars + 6 per lobe."""
    return 15 + LOBE_STRIDE * n_lobes


def round_pitch(n: int, align: int = 32) -> int:
    return max(align, ((n + align - 1) // align) * align)


@dataclasses.dataclass
class Camera:
    R: np.ndarray          # (3,3) float32, world -> camera rotation
    t: np.ndarray          # (3,) float32
    fx: float
    fy: float
    cx: float
    cy: float
    width: int
    height: int
    near: float = 0.2
    bg: tuple = (0.0, 0.0, 0.0)

    @property
    def position(self) -> np.ndarray:
        R = self.R.astype(np.float64)
        return -(R.T @ self.t.astype(np.float64))


@dataclasses.dataclass
class Scene:
    planes: np.ndarray     # (15+6M, pitch) float32
    n: int
    n_lobes: int
    cameras: list
    name: str = ""

    @property
    def pitch(self) -> int:
        return self.planes.shape[1]

    def sha256(self) -> str:
        h = hashlib.sha256()
        h.update(np.ascontiguousarray(self.planes[:, : self.n]).tobytes())
        for c in self.cameras:
            h.update(np.asarray(c.R, np.float32).tobytes())
            h.update(np.asarray(c.t, np.float32).tobytes())
            h.update(np.asarray([c.fx, c.fy, c.cx, c.cy, c.near], np.float32).tobytes())
            h.update(np.asarray([c.width, c.height], np.int32).tobytes())
        return h.hexdigest()


# ----------------------------------------------------------------------------
# cameras
# ----------------------------------------------------------------------------

def look_at(eye, target=(0.0, 0.0, 0.0), up=(0.0, 1.0, 0.0)):
    """World->camera (R, t) for an OpenCV camera at `eye` looking at `target`."""
    eye = np.asarray(eye, np.float64)
    fwd = np.asarray(target, np.float64) - eye
    fwd /= np.linalg.norm(fwd)
    right = np.cross(fwd, np.asarray(up, np.float64))
    if np.linalg.norm(right) < 1e-9:
        right = np.cross(fwd, np.array([0.0, 0.0, 1.0]))
    right /= np.linalg.norm(right)
    down = np.cross(fwd, right)
    R = np.stack([right, down, fwd], axis=0)
    t = -R @ eye
    return R.astype(np.float32), t.astype(np.float32)


def pinhole(R, t, width, height, fov_x_deg=60.0, near=0.2):
    f = (width / 2.0) / math.tan(math.radians(fov_x_deg) / 2.0)
    return Camera(R=np.asarray(R, np.float32), t=np.asarray(t, np.float32),
                  fx=float(np.float32(f)), fy=float(np.float32(f)),
                  cx=width / 2.0, cy=height / 2.0, width=int(width), height=int(height),
                  near=near)


def ring_camera(radius, elev_deg, az, width, height, fov_x_deg=60.0):
    el = math.radians(elev_deg)
    eye = (radius * math.cos(el) * math.sin(az), radius * math.sin(el),
           -radius * math.cos(el) * math.cos(az))
    R, t = look_at(eye)
    return pinhole(R, t, width, height, fov_x_deg)


def ring_cameras(n_views, radius, elev_deg, sizes, fov_x_deg=60.0):
    cams = []
    for k in range(n_views):
        w, h = sizes[k % len(sizes)] if isinstance(sizes, list) else sizes
        cams.append(ring_camera(radius, elev_deg, 2.0 * math.pi * k / n_views, w, h, fov_x_deg))
    return cams


# ----------------------------------------------------------------------------
# primitive draws
# ----------------------------------------------------------------------------

def _unit_quats(rng, n):
    q = rng.standard_normal((n, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    return q


def _lobes(rng, n, n_lobes, planes):
    for m in range(n_lobes):
        base = P_LOBES + LOBE_STRIDE * m
        planes[base + 0, :n] = np.arccos(rng.uniform(-1.0, 1.0, n))       # theta
        planes[base + 1, :n] = rng.uniform(0.0, 2.0 * math.pi, n)          # phi
        planes[base + 2, :n] = rng.normal(0.0, 0.5, n)                      # b_m
        planes[base + 3: base + 6, :n] = rng.uniform(0.0, 0.5, (3, n))      # c_m


def _alloc(n, n_lobes, pitch=None):
    pitch = pitch or round_pitch(n)
    planes = np.zeros((n_planes(n_lobes), pitch), np.float32)
    planes[P_QUAT, :] = 1.0          # padding lanes hold a valid identity rotation
    return planes


def _rot_to_quat(Rm):
    """Rotation matrices (n,3,3) -> unit quaternions (n,4) w,x,y,z."""
    n = Rm.shape[0]
    q = np.empty((n, 4))
    tr = Rm[:, 0, 0] + Rm[:, 1, 1] + Rm[:, 2, 2]
    w = np.sqrt(np.maximum(0.0, 1.0 + tr)) / 2.0
    x = np.sqrt(np.maximum(0.0, 1.0 + Rm[:, 0, 0] - Rm[:, 1, 1] - Rm[:, 2, 2])) / 2.0
    y = np.sqrt(np.maximum(0.0, 1.0 - Rm[:, 0, 0] + Rm[:, 1, 1] - Rm[:, 2, 2])) / 2.0
    z = np.sqrt(np.maximum(0.0, 1.0 - Rm[:, 0, 0] - Rm[:, 1, 1] + Rm[:, 2, 2])) / 2.0
    x = np.copysign(x, Rm[:, 2, 1] - Rm[:, 1, 2])
    y = np.copysign(y, Rm[:, 0, 2] - Rm[:, 2, 0])
    z = np.copysign(z, Rm[:, 1, 0] - Rm[:, 0, 1])
    q[:, 0], q[:, 1], q[:, 2], q[:, 3] = w, x, y, z
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    return q


def random_scene(n, n_lobes, rng, mean_lo=-1.0, mean_hi=1.0, logscale=(-3.5, 0.4),
                 opacity_sd=1.0, b_sd=0.5):
    """Uniform cube of primitives (the 4,096-Beta 256x256 recipe)."""
    planes = _alloc(n, n_lobes)
    planes[P_MEAN:P_MEAN + 3, :n] = rng.uniform(mean_lo, mean_hi, (3, n))
    planes[P_LOGSCALE:P_LOGSCALE + 3, :n] = rng.normal(logscale[0], logscale[1], (3, n))
    planes[P_QUAT:P_QUAT + 4, :n] = _unit_quats(rng, n).T
    planes[P_OPACITY, :n] = rng.normal(0.0, opacity_sd, n)
    planes[P_B, :n] = rng.normal(0.0, b_sd, n)
    planes[P_C0:P_C0 + 3, :n] = rng.uniform(0.0, 1.0, (3, n))
    _lobes(rng, n, n_lobes, planes)
    return planes


def gmm_scene(n, n_lobes, rng, k=64, box=2.0):
    """64-component Gaussian mixture in [-2,2]^3 (the 200k-Beta recipe)."""
    planes = _alloc(n, n_lobes)
    centres = rng.uniform(-box, box, (k, 3))
    sig = rng.uniform(0.05, 0.3, k)
    comp = rng.integers(0, k, n)
    pts = centres[comp] + sig[comp, None] * rng.standard_normal((n, 3))
    planes[P_MEAN:P_MEAN + 3, :n] = np.clip(pts, -box, box).T
    planes[P_LOGSCALE:P_LOGSCALE + 3, :n] = rng.normal(-4.5, 0.5, (3, n))
    planes[P_QUAT:P_QUAT + 4, :n] = _unit_quats(rng, n).T
    planes[P_OPACITY, :n] = rng.normal(0.0, 1.5, n)
    planes[P_B, :n] = rng.normal(0.0, 0.7, n)
    planes[P_C0:P_C0 + 3, :n] = rng.uniform(0.0, 1.0, (3, n))
    _lobes(rng, n, n_lobes, planes)
    return planes


def sheet_scene(n, n_lobes, rng, n_sheets=256):
    """Clustered planar sheets (the 1M/3M/6M-Beta recipe).

    Sheet centre U[-1.5,1.5]^3, normal uniform on the sphere, disk radius
    U[0.3,0.8]; points uniform on the disk plus N(0, 0.005) normal jitter;
    log-scales N(-5, 0.6) with the normal axis (local z) 10x thinner;
    rotation = sheet frame x random in-plane twist.
    """
    planes = _alloc(n, n_lobes)
    centre = rng.uniform(-1.5, 1.5, (n_sheets, 3))
    normal = rng.standard_normal((n_sheets, 3))
    normal /= np.linalg.norm(normal, axis=1, keepdims=True)
    radius = rng.uniform(0.3, 0.8, n_sheets)
    helper = np.where(np.abs(normal[:, :1]) < 0.9, np.array([[1.0, 0.0, 0.0]]), np.array([[0.0, 1.0, 0.0]]))
    e1 = np.cross(normal, helper)
    e1 /= np.linalg.norm(e1, axis=1, keepdims=True)
    e2 = np.cross(normal, e1)
    sheet = rng.integers(0, n_sheets, n)
    rho = np.sqrt(rng.uniform(0.0, 1.0, n)) * radius[sheet]
    ang = rng.uniform(0.0, 2.0 * math.pi, n)
    pos = (centre[sheet] + (rho * np.cos(ang))[:, None] * e1[sheet]
           + (rho * np.sin(ang))[:, None] * e2[sheet]
           + rng.normal(0.0, 0.005, n)[:, None] * normal[sheet])
    planes[P_MEAN:P_MEAN + 3, :n] = pos.T
    ls = rng.normal(-5.0, 0.6, (3, n))
    ls[2] -= math.log(10.0)
    planes[P_LOGSCALE:P_LOGSCALE + 3, :n] = ls
    tw = rng.uniform(0.0, 2.0 * math.pi, n)
    u = np.cos(tw)[:, None] * e1[sheet] + np.sin(tw)[:, None] * e2[sheet]
    v = -np.sin(tw)[:, None] * e1[sheet] + np.cos(tw)[:, None] * e2[sheet]
    Rm = np.stack([u, v, normal[sheet]], axis=2)     # columns: local x, y, z
    planes[P_QUAT:P_QUAT + 4, :n] = _rot_to_quat(Rm).T
    planes[P_OPACITY, :n] = rng.normal(0.0, 1.5, n)
    planes[P_B, :n] = rng.normal(0.0, 0.7, n)
    planes[P_C0:P_C0 + 3, :n] = rng.uniform(0.0, 1.0, (3, n))
    _lobes(rng, n, n_lobes, planes)
    return planes


# ----------------------------------------------------------------------------
# the five workloads
# ----------------------------------------------------------------------------

MIXED_SIZES = [(640, 480), (1280, 720), (1920, 1080), (2560, 1440)]


def workload_sizes(config_id: int, n_views: int, size=None) -> list:
    """(width, height) of each ring view of a workload: 1920x1080 (3), four
    views each of MIXED_SIZES in turn (4), 3840x2160 (5); `size` overrides."""
    if size is not None:
        return [tuple(size)] * n_views
    if config_id == 4:
        return [MIXED_SIZES[k // 4 % 4] for k in range(n_views)]
    if config_id == 5:
        return [(3840, 2160)] * n_views
    return [(1920, 1080)] * n_views


def describe_sizes(cams) -> str:
    """'1920x1080' for equal views, else the count of each size."""
    sizes = [(c.width, c.height) for c in cams]
    if len(set(sizes)) == 1:
        return f"{sizes[0][0]}x{sizes[0][1]}"
    out = []
    for wh in sorted(set(sizes)):
        out.append(f"{sizes.count(wh)} x {wh[0]}x{wh[1]}")
    return "mixed (" + ", ".join(out) + ")"


def config_scene(config_id: int, n: int | None = None, n_views: int | None = None,
                 seed: int | None = None) -> Scene:
    """Workloads of the benchmark table, with optional down-scaled primitive counts.

    1: 4,096 Betas, 256x256, camera at (0,0,-3), 1 lobe, forward only
    2: 200k Betas (Gaussian mixture), 1297x840, 2 lobes, forward + backward
    3: 1M Betas (256 sheets), 1920x1080, 3 lobes, 16 ring views, view 0 timed
    4: 3M Betas (sheets), 16 views of mixed resolution, 3 lobes
    5: 6M Betas (sheets), 8 views of 3840x2160, 3 lobes
    """
    rng = np.random.Generator(np.random.PCG64((SEED_BASE + config_id) if seed is None else seed))
    if config_id == 1:
        n = n or 4096
        planes = random_scene(n, 1, rng)
        R, t = look_at((0.0, 0.0, -3.0))
        cams = [pinhole(R, t, 256, 256)]
        m = 1
    elif config_id == 2:
        n = n or 200_000
        planes = gmm_scene(n, 2, rng)
        cams = [ring_camera(4.0, 20.0, 0.0, 1297, 840)]
        m = 2
    elif config_id == 3:
        n = n or 1_000_000
        planes = sheet_scene(n, 3, rng)
        cams = ring_cameras(n_views or 16, 4.0, 15.0, (1920, 1080))
        m = 3
    elif config_id == 4:
        n = n or 3_000_000
        planes = sheet_scene(n, 3, rng)
        nv = n_views or 16
        sizes = [MIXED_SIZES[k // 4 % 4] for k in range(nv)]
        cams = [ring_camera(4.0, 15.0, 2.0 * math.pi * k / nv, w, h) for k, (w, h) in enumerate(sizes)]
        m = 3
    elif config_id == 5:
        n = n or 6_000_000
        planes = sheet_scene(n, 3, rng)
        cams = ring_cameras(n_views or 8, 4.0, 15.0, (3840, 2160))
        m = 3
    else:
        raise ValueError(f"unknown workload {config_id}")
    return Scene(planes=planes, n=n, n_lobes=m, cameras=cams, name=f"workload{config_id}")


def target_images(cameras, seed: int):
    """Seeded U[0,1] target images, one (3,H,W) float32 array per camera."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return [rng.uniform(0.0, 1.0, (3, c.height, c.width)).astype(np.float32) for c in cameras]


def sample_pixels(camera, count: int, seed: int, full_tiles: int = 0, tile: int = 16):
    """Seeded pixel sample: `count` random pixels plus `full_tiles` whole tiles.

    Returns (xs, ys) int32 arrays, without duplicates.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    W, H = camera.width, camera.height
    idx = rng.choice(W * H, size=min(count, W * H), replace=False)
    xs, ys = list(idx % W), list(idx // W)
    ntx, nty = (W + tile - 1) // tile, (H + tile - 1) // tile
    for t in rng.choice(ntx * nty, size=min(full_tiles, ntx * nty), replace=False):
        tx, ty = t % ntx, t // ntx
        for yy in range(ty * tile, min(H, ty * tile + tile)):
            for xx in range(tx * tile, min(W, tx * tile + tile)):
                xs.append(xx)
                ys.append(yy)
    pix = np.unique(np.asarray(ys, np.int64) * W + np.asarray(xs, np.int64))
    return (pix % W).astype(np.int32), (pix // W).astype(np.int32)
