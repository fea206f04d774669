"""Hand-built primitives and cameras for the closed-form tests."""
import math

import numpy as np

from paper_2501_18630_gb300 import scenes


def logit(o):
    return math.log(o / (1.0 - o))


def prim(mu=(0.0, 0.0, 5.0), scale=(0.1, 0.1, 0.1), quat=(1.0, 0.0, 0.0, 0.0), opacity=0.5,
         b=0.0, c0=(0.2, 0.5, 0.9), lobes=()):
    """One primitive as a dict of raw parameters (scale given linearly)."""
    return dict(mu=mu, logscale=tuple(math.log(s) for s in scale), quat=quat,
                ologit=logit(opacity), b=b, c0=c0, lobes=tuple(lobes))


def planes_of(prims, n_lobes=0, pitch=None):
    n = len(prims)
    pitch = pitch or scenes.round_pitch(max(n, 1))
    P = np.zeros((scenes.n_planes(n_lobes), pitch), np.float32)
    P[scenes.P_QUAT, :] = 1.0
    for i, p in enumerate(prims):
        P[0:3, i] = p["mu"]
        P[3:6, i] = p["logscale"]
        P[6:10, i] = p["quat"]
        P[10, i] = p["ologit"]
        P[11, i] = p["b"]
        P[12:15, i] = p["c0"]
        for m, lob in enumerate(p["lobes"]):
            P[15 + 6 * m: 21 + 6 * m, i] = lob
    return P


def axis_camera(width=33, height=33, f=100.0, cx=16.5, cy=16.5, R=None, t=None, bg=(0.0, 0.0, 0.0)):
    """Camera at the origin looking down +z (identity pose) unless R, t given."""
    R = np.eye(3, dtype=np.float32) if R is None else np.asarray(R, np.float32)
    t = np.zeros(3, np.float32) if t is None else np.asarray(t, np.float32)
    return scenes.Camera(R=R, t=t, fx=f, fy=f, cx=cx, cy=cy, width=width, height=height, near=0.2, bg=bg)


def f32(x):
    return float(np.float32(x))


def quat_mul(a, b):
    """Hamilton product a*b of (w,x,y,z) quaternions."""
    aw, ax, ay, az = a
    bw, bx, by, bz = b
    return (aw * bw - ax * bx - ay * by - az * bz,
            aw * bx + ax * bw + ay * bz - az * by,
            aw * by - ax * bz + ay * bw + az * bx,
            aw * bz + ax * by - ay * bx + az * bw)


def axis_angle_quat(axis, ang):
    axis = np.asarray(axis, np.float64)
    axis = axis / np.linalg.norm(axis)
    s = math.sin(ang / 2.0)
    return (math.cos(ang / 2.0), axis[0] * s, axis[1] * s, axis[2] * s)


def axis_angle_matrix(axis, ang):
    """Rodrigues' formula, independent of any quaternion code."""
    k = np.asarray(axis, np.float64)
    k = k / np.linalg.norm(k)
    K = np.array([[0, -k[2], k[1]], [k[2], 0, -k[0]], [-k[1], k[0], 0]])
    return np.eye(3) + math.sin(ang) * K + (1 - math.cos(ang)) * (K @ K)
