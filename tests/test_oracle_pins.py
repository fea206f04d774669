"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test derives its expected value independently of the oracle's general
code path: closed forms of special cases, invariances, the densification
identity of Appendix C, and brute force on tiny inputs.
"""
import json
import math
import os

import numpy as np
import pytest

import oracle
from paper_2501_18630_gb300 import scenes
from tests.helpers import (axis_angle_matrix, axis_angle_quat, axis_camera, f32, logit,
                           planes_of, prim, quat_mul)

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def eff(p):
    """Effective (fp32-stored) opacity, beta and linear scales of a prim dict."""
    o = 1.0 / (1.0 + math.exp(-f32(p["ologit"])))
    beta = 4.0 * math.exp(f32(p["b"]))
    s = [math.exp(f32(v)) for v in p["logscale"]]
    return o, beta, s


def render1(prims, cam, xs, ys, n_lobes=0, **kw):
    P = planes_of(prims, n_lobes)
    return oracle.render(P, len(prims), n_lobes, cam, np.asarray(xs), np.asarray(ys), **kw)


# --------------------------------------------------------------------------
# Beta kernel and a single splat (Eq. 2, Eq. eq:beta, Eq. r, Eq. C)
# --------------------------------------------------------------------------

def test_single_splat_centre_closed_form():
    """At the projected centre r = 0, B = 1, so C = c o and T = 1 - o."""
    p = prim(mu=(0.0, 0.0, 5.0), scale=(0.2, 0.2, 0.2), opacity=0.7, b=0.3, c0=(0.2, 0.5, 0.9))
    cam = axis_camera()
    C, T, last, cnt = render1([p], cam, [16], [16])
    o, _, _ = eff(p)
    assert np.allclose(C[0], np.array([f32(v) for v in p["c0"]]) * o, rtol=0, atol=1e-15)
    assert abs(T[0] - (1.0 - o)) < 1e-15
    assert last[0] == 0 and cnt[0] == 1


@pytest.mark.parametrize("b", [-1.5, 0.0, 0.8, 2.0])
def test_isotropic_radial_profile(b):
    """Sphere on the optical axis: Sigma' = (f s / z)^2 I, so along a pixel row
    alpha = o (1 - (d/rho)^2)^(4 e^b) inside rho = f s / z and 0 outside."""
    z, f = 5.0, 100.0
    p = prim(mu=(0.0, 0.0, z), scale=(0.225, 0.225, 0.225), opacity=0.6, b=b, c0=(1.0, 1.0, 1.0))
    cam = axis_camera(width=40, f=f)
    xs = np.arange(16, 40)
    C, T, last, _ = render1([p], cam, xs, np.full_like(xs, 16))
    o, beta, s = eff(p)
    rho = f * s[0] / z
    for k, x in enumerate(xs):
        d = (x + 0.5) - 16.5
        r2 = (d / rho) ** 2
        a = o * (1.0 - r2) ** beta if r2 < 1.0 else 0.0
        assert abs((1.0 - T[k]) - a) < 1e-13, (x, r2)
        assert abs(C[k, 0] - a) < 1e-13
        assert (last[k] == 0) == (r2 < 1.0)


def test_beta_reparameterisation_b0_is_4():
    """b = 0 gives beta = 4 (Eq. eq:beta): alpha(r) = o (1 - r^2)^4."""
    p = prim(scale=(0.2, 0.2, 0.2), opacity=0.5, b=0.0, c0=(1, 1, 1))
    cam = axis_camera(width=40)
    C, T, _, _ = render1([p], cam, [18], [16])
    o, _, s = eff(p)
    r2 = (2.0 / (100.0 * s[0] / 5.0)) ** 2
    assert abs((1 - T[0]) - o * (1 - r2) ** 4) < 1e-14


def test_anisotropic_axes_and_rotations():
    """Axis-aligned ellipsoid at the axis: Sigma' = diag((f sx/z)^2, (f sy/z)^2).
    A 90 degree turn about z swaps the x and y extents; one about y puts sz on x."""
    z, f = 5.0, 100.0
    sc = (0.3, 0.15, 0.05)
    cam = axis_camera(width=33, f=f)
    xs = np.array([16, 17, 18, 19, 20, 16, 16, 16])
    ys = np.array([16, 16, 16, 16, 16, 17, 18, 19])
    for quat, (ex_s, ey_s) in [((1, 0, 0, 0), (sc[0], sc[1])),
                               (axis_angle_quat((0, 0, 1), math.pi / 2), (sc[1], sc[0])),
                               (axis_angle_quat((0, 1, 0), math.pi / 2), (sc[2], sc[1]))]:
        p = prim(mu=(0.0, 0.0, z), scale=sc, quat=quat, opacity=0.5, b=0.0, c0=(1, 1, 1))
        o, beta, s = eff(p)
        sx = s[0] if ex_s == sc[0] else (s[1] if ex_s == sc[1] else s[2])
        sy = s[0] if ey_s == sc[0] else (s[1] if ey_s == sc[1] else s[2])
        C, T, _, _ = render1([p], cam, xs, ys)
        for k in range(len(xs)):
            dx, dy = xs[k] - 16, ys[k] - 16
            r2 = (dx / (f * sx / z)) ** 2 + (dy / (f * sy / z)) ** 2
            a = o * (1 - r2) ** beta if r2 < 1 else 0.0
            assert abs((1 - T[k]) - a) < 1e-7, (quat, xs[k], ys[k])


def test_off_axis_centre_and_jacobian():
    """mu' = (f x/z + cx, f y/z + cy); for a sphere Sigma' = (f s/z)^2 (I + u u^T)
    with u = (x/z, y/z): the closed form of J J^T s^2."""
    f, z, X, Y = 100.0, 4.0, 0.4, -0.2          # mu' = (26.5, 11.5)
    p = prim(mu=(X, Y, z), scale=(0.1, 0.1, 0.1), opacity=0.8, b=0.5, c0=(0.3, 0.6, 0.9))
    cam = axis_camera(width=40, height=40, f=f)
    o, beta, s = eff(p)
    C, T, _, _ = render1([p], cam, [26], [11])
    assert abs((1 - T[0]) - o) < 1e-13
    u = np.array([f32(X) / f32(z), f32(Y) / f32(z)])
    cov = (f * s[0] / f32(z)) ** 2 * (np.eye(2) + np.outer(u, u))
    Q = np.linalg.inv(cov)
    xs = np.array([27, 28, 25, 26, 27, 24])
    ys = np.array([11, 12, 10, 13, 9, 11])
    mu2 = np.array([f * f32(X) / f32(z) + 16.5, f * f32(Y) / f32(z) + 16.5])
    C, T, _, _ = render1([p], cam, xs, ys)
    for k in range(len(xs)):
        d = np.array([xs[k] + 0.5, ys[k] + 0.5]) - mu2
        r2 = d @ Q @ d
        a = o * (1 - r2) ** beta if r2 < 1 else 0.0
        assert abs((1 - T[k]) - a) < 1e-12


def test_projected_silhouette_matches_support():
    """Independent geometric pin of Sigma' = J W R S S^T R^T W^T J^T: sample the
    3D support ellipsoid {mu + R S u : |u| = 1}, project every point through
    the exact pinhole, and evaluate the oracle's r^2 there.  The EWA
    linearisation makes the silhouette the r^2 = 1 contour up to O(size/depth)."""
    rng = np.random.default_rng(0)
    Rw = axis_angle_matrix((0.3, 1.0, -0.2), 0.4).astype(np.float32)
    tw = np.array([0.1, -0.2, 0.3], np.float32)
    cam = scenes.Camera(R=Rw, t=tw, fx=900.0, fy=700.0, cx=250.0, cy=180.0, width=500, height=400)
    for trial in range(5):
        q = rng.standard_normal(4)
        q /= np.linalg.norm(q)
        sc = np.exp(rng.normal(-5.0, 0.5, 3))
        cam_pt = np.array([rng.uniform(-1, 1), rng.uniform(-0.8, 0.8), rng.uniform(5, 8)])
        mu = (Rw.astype(np.float64).T @ (cam_pt - tw.astype(np.float64)))
        p = prim(mu=tuple(mu), scale=tuple(sc), quat=tuple(q), opacity=0.5)
        P = planes_of([p])
        pr = oracle.project(P, 1, 0, cam)
        A, B, Cc = pr["conic"][0]
        mu2 = pr["mu2"][0]
        # rotation by Rodrigues from the axis-angle of q (independent of the oracle's formula)
        qf = P[6:10, 0].astype(np.float64)
        qf /= np.linalg.norm(qf)
        ang = 2 * math.acos(max(-1.0, min(1.0, qf[0])))
        Rq = axis_angle_matrix(qf[1:], ang) if ang > 1e-12 else np.eye(3)
        s = np.exp(P[3:6, 0].astype(np.float64))
        u = rng.standard_normal((20000, 3))
        u /= np.linalg.norm(u, axis=1, keepdims=True)
        pts = P[0:3, 0].astype(np.float64) + (u * s) @ Rq.T
        cpts = pts @ Rw.astype(np.float64).T + tw.astype(np.float64)
        px = cam.fx * cpts[:, 0] / cpts[:, 2] + cam.cx
        py = cam.fy * cpts[:, 1] / cpts[:, 2] + cam.cy
        dx, dy = px - mu2[0], py - mu2[1]
        r2 = A * dx * dx + 2 * B * dx * dy + Cc * dy * dy
        tol = 6 * s.max() / cam_pt[2]
        assert abs(r2.max() - 1.0) < tol, (trial, r2.max(), tol)


# --------------------------------------------------------------------------
# depth ordering and compositing (Sec. 3.2, Eq. C)
# --------------------------------------------------------------------------

def test_two_splats_front_to_back_closed_form():
    """C = c1 a1 + c2 a2 (1 - a1), with 1 the nearer splat, whatever the index order."""
    near = prim(mu=(0.0, 0.0, 4.0), scale=(0.2,) * 3, opacity=0.6, c0=(1.0, 0.0, 0.0))
    far = prim(mu=(0.0, 0.0, 6.0), scale=(0.3,) * 3, opacity=0.5, c0=(0.0, 0.0, 1.0))
    cam = axis_camera()
    on, _, _ = eff(near)
    of, _, _ = eff(far)
    for order in ([near, far], [far, near]):
        C, T, last, cnt = render1(order, cam, [16], [16])
        assert abs(C[0, 0] - on) < 1e-15
        assert abs(C[0, 2] - of * (1 - on)) < 1e-15
        assert abs(T[0] - (1 - on) * (1 - of)) < 1e-15
        assert cnt[0] == 2
        assert order[last[0]] is far            # the far splat is composited last


def test_equal_depth_ties_by_index():
    a = prim(mu=(0.0, 0.0, 5.0), scale=(0.2,) * 3, opacity=0.4, c0=(1.0, 0.0, 0.0))
    b = prim(mu=(0.0, 0.0, 5.0), scale=(0.2,) * 3, opacity=0.4, c0=(0.0, 1.0, 0.0))
    C, T, last, _ = render1([a, b], axis_camera(), [16], [16])
    o, _, _ = eff(a)
    assert abs(C[0, 0] - o) < 1e-15 and abs(C[0, 1] - o * (1 - o)) < 1e-15
    assert last[0] == 1


def test_disjoint_splats_are_order_independent_and_additive():
    rng = np.random.default_rng(3)
    prims = [prim(mu=(x, y, z), scale=(0.15, 0.12, 0.1), quat=tuple(rng.standard_normal(4)),
                  opacity=0.7, b=rng.normal(0, 0.5), c0=tuple(rng.uniform(0, 1, 3)))
             for x, y, z in [(-0.6, -0.6, 5.0), (0.6, -0.5, 5.5), (0.0, 0.6, 4.5)]]
    cam = axis_camera(width=64, height=64, cx=32, cy=32)
    full = oracle.render_full(planes_of(prims), 3, 0, cam)
    acc = np.zeros((3, 64, 64))
    Tprod = np.ones((64, 64))
    for p in prims:
        C, T, _, _ = oracle.render_full(planes_of([p]), 1, 0, cam)
        acc += C
        Tprod *= T
        assert (T < 1).sum() > 10
    assert np.abs(full[0] - acc).max() < 1e-15
    assert np.abs(full[1] - Tprod).max() < 1e-15
    rev = oracle.render_full(planes_of(prims[::-1]), 3, 0, cam)
    assert np.abs(rev[0] - full[0]).max() < 1e-15


def test_alpha_clamp():
    p = prim(scale=(0.2,) * 3, opacity=0.999, c0=(1, 1, 1))
    C, T, _, _ = render1([p], axis_camera(), [16], [16])
    assert abs(T[0] - (1 - f32(0.99))) < 1e-15   # options are fp32, as on the GPU
    C2, T2, _, _ = render1([p], axis_camera(), [16], [16], alpha_max=0.995)
    assert abs(T2[0] - (1 - f32(0.995))) < 1e-15


def test_early_termination_rule():
    """Stop before primitive k once T < t_eps: three clamped layers leave
    T = 0.01^3 = 1e-6 < 2^-19, so the fourth layer is never composited."""
    layers = [prim(mu=(0.0, 0.0, 4.0 + k), scale=(0.2 * (4 + k) / 4,) * 3, opacity=0.9999,
                   c0=(0.1 * (k + 1), 0.0, 0.0)) for k in range(5)]
    C, T, last, cnt = render1(layers, axis_camera(), [16], [16])
    assert cnt[0] == 3 and last[0] == 2
    a = f32(0.99)
    expect = f32(0.1) * a + f32(0.2) * a * (1 - a) + f32(0.3) * a * (1 - a) ** 2
    assert abs(C[0, 0] - expect) < 1e-12
    C, T, last, cnt = render1(layers, axis_camera(), [16], [16], t_eps=1e-7)
    assert cnt[0] == 4


def test_background_weighted_by_final_transmittance():
    p = prim(scale=(0.2,) * 3, opacity=0.3, c0=(0.0, 0.0, 0.0))
    cam = axis_camera(bg=(0.25, 0.5, 1.0))
    C, T, _, _ = render1([p], cam, [16, 0], [16, 0])
    o, _, _ = eff(p)
    assert np.allclose(C[0], (1 - o) * np.array([0.25, 0.5, 1.0]), atol=1e-15)
    assert np.allclose(C[1], [0.25, 0.5, 1.0], atol=0) and T[1] == 1.0


# --------------------------------------------------------------------------
# opacity-only relocation (Sec. 3.4, Appendix C, Eq. eq:densify)
# --------------------------------------------------------------------------

@pytest.mark.parametrize("N", [2, 3, 5])
def test_relocation_identity_exact_at_centre(N):
    """N coincident clones with o' = 1 - (1 - o)^(1/N) give total alpha o at the
    centre exactly (f = 1 there)."""
    o = 0.3
    op = 1.0 - (1.0 - o) ** (1.0 / N)
    clones = [prim(mu=(0.0, 0.0, 5.0), scale=(0.2,) * 3, opacity=op, b=0.2, c0=(1, 1, 1))] * N
    C, T, _, cnt = render1(clones, axis_camera(), [16], [16])
    o_eff = 1.0 / (1.0 + math.exp(-f32(logit(op))))
    assert cnt[0] == N
    assert abs((1 - T[0]) - (1 - (1 - o_eff) ** N)) < 1e-15
    assert abs((1 - T[0]) - o) < 5e-7      # fp32 storage of the opacity logit


def test_relocation_off_centre_error_is_second_order():
    """Off-centre the clones give 1 - (1 - o' f)^N instead of o f; the gap is
    O(o^2) (Appendix C): halving o divides it by about four."""
    N = 4
    gaps = []
    for o in (0.2, 0.1, 0.05):
        op = 1.0 - (1.0 - o) ** (1.0 / N)
        single = prim(scale=(0.2,) * 3, opacity=o, b=0.0, c0=(1, 1, 1))
        clones = [prim(scale=(0.2,) * 3, opacity=op, b=0.0, c0=(1, 1, 1))] * N
        xs = np.array([17, 18, 19])
        _, T1, _, _ = render1([single], axis_camera(width=40), xs, np.full(3, 16))
        _, TN, _, _ = render1(clones, axis_camera(width=40), xs, np.full(3, 16))
        gap = np.abs((1 - TN) - (1 - T1))
        gaps.append(gap.max())
        assert gap.max() < o * o
    assert 3.0 < gaps[0] / gaps[1] < 5.0 and 3.0 < gaps[1] / gaps[2] < 5.0


# --------------------------------------------------------------------------
# spherical Beta colour (Sec. 3.3)
# --------------------------------------------------------------------------

def sb_prim(theta, phi, bm, cm=(0.4, 0.3, 0.2), c0=(0.1, 0.2, 0.3)):
    return prim(mu=(0.0, 0.0, 5.0), scale=(0.2,) * 3, opacity=0.5, c0=c0,
                lobes=[(theta, phi, bm) + tuple(cm)])


def colour_at_centre(p, n_lobes=1, color_mode=0):
    C, T, _, _ = render1([p], axis_camera(), [16], [16], n_lobes=n_lobes, color_mode=color_mode)
    o, _, _ = eff(p)
    return C[0] / o


def test_sb_lobe_aligned_with_view_adds_full_colour():
    """R_m = V (theta = 0 for a splat on the +z axis seen from the origin):
    B(1 - 1; b_m) = 1, so c = c0 + c_m for any b_m."""
    for bm in (-1.0, 0.0, 1.5):
        c = colour_at_centre(sb_prim(0.0, 0.0, bm))
        assert np.allclose(c, np.array([0.1 + 0.4, 0.2 + 0.3, 0.3 + 0.2], np.float32), atol=1e-7)


def test_sb_lobe_zero_when_back_facing_and_continuous_at_orthogonal():
    c0 = np.array([0.1, 0.2, 0.3], np.float32)
    for theta in (math.pi, 2.5, math.pi / 2 + 1e-3):
        assert np.allclose(colour_at_centre(sb_prim(theta, 0.7, 0.0)), c0, atol=1e-7)
    near_orth = colour_at_centre(sb_prim(math.pi / 2 - 1e-3, 0.0, 0.0))
    assert np.abs(near_orth - c0).max() < 1e-10


def test_sb_lobe_intermediate_angle():
    """R.V = cos(theta) for a splat on the axis: term = cos(theta)^(4 e^b_m)."""
    theta, bm = 0.6, 0.4
    c = colour_at_centre(sb_prim(theta, 1.1, bm))
    w = math.cos(f32(theta)) ** (4 * math.exp(f32(bm)))
    assert np.allclose(c, np.array([0.1, 0.2, 0.3]) + w * np.array([0.4, 0.3, 0.2]), atol=1e-7)


def test_sb_phi_rotates_lobe_about_z():
    """A splat off-axis at +x: V has a +x component; the lobe with phi = 0 tilts
    towards it, phi = pi tilts away."""
    p0 = prim(mu=(1.0, 0.0, 5.0), scale=(0.2,) * 3, opacity=0.5, c0=(0, 0, 0), lobes=[(0.5, 0.0, 0.0, 1, 1, 1)])
    p1 = prim(mu=(1.0, 0.0, 5.0), scale=(0.2,) * 3, opacity=0.5, c0=(0, 0, 0), lobes=[(0.5, math.pi, 0.0, 1, 1, 1)])
    cam = axis_camera(width=60, f=100.0)   # mu' = (36.5, 16.5)
    V = np.array([1.0, 0.0, 5.0]) / math.sqrt(26.0)
    for p, phi in ((p0, 0.0), (p1, math.pi)):
        C, T, _, _ = render1([p], cam, [36], [16], n_lobes=1)
        o, _, _ = eff(p)
        Rm = np.array([math.sin(0.5) * math.cos(phi), math.sin(0.5) * math.sin(phi), math.cos(0.5)])
        assert abs(C[0, 0] / o - max(Rm @ V, 0) ** 4) < 1e-6


def test_colour_modes():
    p = sb_prim(0.0, 0.0, 0.0)
    full = colour_at_centre(p, color_mode=0)
    diff = colour_at_centre(p, color_mode=1)
    spec = colour_at_centre(p, color_mode=2)
    assert np.allclose(diff, [0.1, 0.2, 0.3], atol=1e-7)
    assert np.allclose(spec, [0.4, 0.3, 0.2], atol=1e-7)
    assert np.allclose(full, diff + spec, atol=1e-7)


# --------------------------------------------------------------------------
# invariances of the projection
# --------------------------------------------------------------------------

def test_quaternion_sign_and_scale_invariance():
    rng = np.random.default_rng(1)
    q = tuple(rng.standard_normal(4))
    base = prim(scale=(0.3, 0.1, 0.05), quat=q, opacity=0.6, b=0.3)
    cam = axis_camera(width=40, height=40, cx=20, cy=20)
    ref = oracle.render_full(planes_of([base]), 1, 0, cam)[0]
    for q2 in (tuple(-v for v in q), tuple(2.0 * v for v in q), tuple(0.25 * v for v in q)):  # exact in fp32
        p = dict(base, quat=q2)
        img = oracle.render_full(planes_of([p]), 1, 0, cam)[0]
        assert np.abs(img - ref).max() < 1e-12


def test_rigid_motion_invariance():
    """Moving the world by G and the camera by G^-1 leaves the image unchanged
    (the scene is rotated with quaternion products, the camera with matrices)."""
    rng = np.random.default_rng(2)
    G = axis_angle_matrix((1.0, 2.0, 0.5), 0.8)
    qG = axis_angle_quat((1.0, 2.0, 0.5), 0.8)
    shift = np.array([0.25, -0.5, 0.75])
    prims, moved = [], []
    for k in range(4):
        mu = np.array([rng.uniform(-0.5, 0.5), rng.uniform(-0.5, 0.5), rng.uniform(4, 6)])
        q = tuple(rng.standard_normal(4))
        th, ph = 0.4 + 0.3 * k, 0.5 * k
        Rm = np.array([math.sin(th) * math.cos(ph), math.sin(th) * math.sin(ph), math.cos(th)])
        Rm2 = G @ Rm
        kw = dict(scale=tuple(np.exp(rng.normal(-3, 0.3, 3))), opacity=0.5, b=rng.normal(0, 0.5),
                  c0=tuple(rng.uniform(0, 1, 3)))
        prims.append(prim(mu=tuple(mu), quat=q, lobes=[(th, ph, 0.3, 0.5, 0.4, 0.3)], **kw))
        moved.append(prim(mu=tuple(G @ mu + shift), quat=quat_mul(qG, q),
                          lobes=[(math.acos(Rm2[2]), math.atan2(Rm2[1], Rm2[0]), 0.3, 0.5, 0.4, 0.3)], **kw))
    cam = axis_camera(width=48, height=48, cx=24, cy=24)
    # camera for the moved world: x_cam = G^T (x - shift)
    cam2 = axis_camera(width=48, height=48, cx=24, cy=24, R=G.T, t=-(G.T @ shift))
    a = oracle.render_full(planes_of(prims, 1), 4, 1, cam)
    b = oracle.render_full(planes_of(moved, 1), 4, 1, cam2)
    # fp32 storage of the moved inputs perturbs the centres by ~1e-7 relative
    assert np.abs(a[0] - b[0]).max() < 2e-4
    assert (a[3] == b[3]).mean() > 0.99


def test_threads_do_not_change_results():
    sc = scenes.config_scene(1, n=512)
    cam = sc.cameras[0]
    one = oracle.render_full(sc.planes, sc.n, sc.n_lobes, cam, n_threads=1)
    many = oracle.render_full(sc.planes, sc.n, sc.n_lobes, cam, n_threads=7)
    for x, y in zip(one, many):
        assert np.array_equal(x, y)


def test_brute_force_numpy_renderer_tiny_scene():
    """An independent numpy renderer (matrix inverse, cumulative products) on a
    tiny scene agrees with the C oracle to FP64 rounding."""
    sc = scenes.config_scene(1, n=24, seed=7)
    cam = scenes.pinhole(*scenes.look_at((0.0, 0.0, -3.0)), 40, 32)
    P = sc.planes.astype(np.float64)
    n = sc.n
    Rw, tw = cam.R.astype(np.float64), cam.t.astype(np.float64)
    mu = P[0:3, :n].T
    t = mu @ Rw.T + tw
    s = np.exp(P[3:6, :n].T)
    q = P[6:10, :n].T / np.linalg.norm(P[6:10, :n].T, axis=1, keepdims=True)
    img = np.zeros((cam.height, cam.width, 3))
    Tm = np.ones((cam.height, cam.width))
    depth = np.array([np.float32(((np.float32(Rw[2, 0]) * np.float32(m[0]) + np.float32(Rw[2, 1]) * np.float32(m[1]))
                                  + np.float32(Rw[2, 2]) * np.float32(m[2])) + np.float32(tw[2])) for m in mu.astype(np.float32)])
    order = np.lexsort((np.arange(n), depth))
    ys, xs = np.mgrid[0:cam.height, 0:cam.width] + 0.5
    campos = -Rw.T @ tw
    for i in order:
        ang = 2 * math.acos(max(-1.0, min(1.0, q[i, 0])))
        Rq = axis_angle_matrix(q[i, 1:], ang) if ang > 1e-12 else np.eye(3)
        Sig = Rq @ np.diag(s[i] ** 2) @ Rq.T
        x, y, z = t[i]
        J = np.array([[cam.fx / z, 0, -cam.fx * x / z ** 2], [0, cam.fy / z, -cam.fy * y / z ** 2]])
        cov = J @ Rw @ Sig @ Rw.T @ J.T
        Q = np.linalg.inv(cov)
        m2 = np.array([cam.fx * x / z + cam.cx, cam.fy * y / z + cam.cy])
        dx, dy = xs - m2[0], ys - m2[1]
        r2 = Q[0, 0] * dx * dx + 2 * Q[0, 1] * dx * dy + Q[1, 1] * dy * dy
        o = 1 / (1 + np.exp(-P[10, i]))
        beta = 4 * np.exp(P[11, i])
        a = np.where(r2 < 1, np.minimum(0.99, o * np.clip(1 - r2, 0, None) ** beta), 0.0)
        V = (mu[i] - campos) / np.linalg.norm(mu[i] - campos)
        th, ph, bm = P[15:18, i]
        Rm = np.array([math.sin(th) * math.cos(ph), math.sin(th) * math.sin(ph), math.cos(th)])
        col = P[12:15, i] + max(Rm @ V, 0.0) ** (4 * math.exp(bm)) * P[18:21, i]
        img += (Tm * a)[..., None] * col
        Tm *= 1 - a
    C, T, _, _ = oracle.render_full(sc.planes, sc.n, sc.n_lobes, cam)
    assert np.abs(C.transpose(1, 2, 0) - img).max() < 1e-12
    assert np.abs(T - Tm).max() < 1e-12


# --------------------------------------------------------------------------
# finite differences of the oracle (used as the gradient reference)
# --------------------------------------------------------------------------

def test_fd_gradient_of_single_pixel_closed_form():
    """1x1 image, splat centred on the pixel: C = c o, L = mean_ch |c o - t|, so
    dL/d logit = sum_ch sign(c o - t) c o (1 - o) / 3 and dL/dc_ch = sign * o / 3."""
    p = prim(mu=(0.0, 0.0, 5.0), scale=(0.2,) * 3, opacity=0.6, c0=(0.2, 0.5, 0.9))
    cam = axis_camera(width=1, height=1, cx=0.5, cy=0.5)
    P = planes_of([p])
    target = [np.array([0.0, 1.0, 0.1], np.float32).reshape(3, 1, 1)]
    g, gp, gm = oracle.fd_grad(P, 1, 0, [cam], target, plane_ids=[10, 12, 13, 14], prim_ids=[0], local=False)
    o, _, _ = eff(p)
    c = np.array([f32(v) for v in p["c0"]])
    sgn = np.sign(c * o - target[0].reshape(3))
    assert abs(g[0, 0] - (sgn * c).sum() * o * (1 - o) / 3) < 1e-8
    assert np.allclose(g[1:, 0], sgn * o / 3, atol=1e-8)


def test_fd_local_mode_equals_whole_image():
    """The local finite differences (only the pixels of the perturbed
    primitive's padded FP64 support box re-rendered, the rest of the loss
    cancelling) equal the whole-image differences.  The scene has strongly
    anisotropic splats (a wrong axis in the box misses pixels), a large
    splat covering most of the image, splats cut by each image edge (box
    clipping) and overlapping splats (the other primitives' pixels in the box
    must be rendered with them), in two views."""
    prims = [
        prim(mu=(0.0, 0.0, 4.0), scale=(0.9, 0.6, 0.5), opacity=0.5, b=0.3, c0=(0.6, 0.2, 0.1)),  # large
        prim(mu=(0.3, -0.1, 3.5), scale=(0.35, 0.03, 0.03), opacity=0.8, b=-0.2, c0=(0.1, 0.9, 0.3)),  # wide
        prim(mu=(-0.2, 0.2, 3.0), scale=(0.02, 0.3, 0.02), opacity=0.7, b=0.5, c0=(0.9, 0.9, 0.1)),  # tall
        prim(mu=(1.25, 0.0, 4.0), scale=(0.3, 0.2, 0.2), opacity=0.6, b=0.0, c0=(0.2, 0.3, 0.8)),   # right edge
        prim(mu=(-1.3, -0.4, 4.0), scale=(0.25, 0.3, 0.2), opacity=0.6, b=0.1, c0=(0.7, 0.1, 0.5)),  # left edge
        prim(mu=(0.1, 1.05, 4.2), scale=(0.3, 0.25, 0.2), opacity=0.55, b=-0.1, c0=(0.4, 0.6, 0.2)),  # bottom
        prim(mu=(-0.1, -1.0, 4.1), scale=(0.28, 0.3, 0.2), opacity=0.65, b=0.2, c0=(0.3, 0.2, 0.9)),  # top
        prim(mu=(0.25, 0.05, 3.8), scale=(0.12, 0.12, 0.12), opacity=0.9, b=0.7, c0=(0.5, 0.5, 0.5),
             lobes=[(0.4, 1.0, 0.2, 0.3, 0.1, 0.2)]),
    ]
    for p in prims[:-1]:
        p["lobes"] = ((0.3, 2.0, 0.1, 0.2, 0.2, 0.1),)
    P = planes_of(prims, n_lobes=1)
    q = axis_angle_quat((0.3, 0.2, 1.0), 0.7)
    P[6:10, 1] = q                                         # rotate the wide splat
    cams = [axis_camera(width=48, height=40, f=40.0, cx=24.0, cy=20.0),
            axis_camera(width=37, height=29, f=30.0, cx=17.0, cy=15.5)]
    rng = np.random.default_rng(3)
    targets = [rng.uniform(0, 1, (3, c.height, c.width)).astype(np.float32) for c in cams]
    n = len(prims)
    planes = list(range(scenes.n_planes(1)))
    g_loc, _, _ = oracle.fd_grad(P, n, 1, cams, targets, planes, list(range(n)), local=True)
    g_all, _, _ = oracle.fd_grad(P, n, 1, cams, targets, planes, list(range(n)), local=False)
    scale = np.abs(g_all).max()
    assert scale > 1e-3
    assert np.abs(g_loc - g_all).max() <= 1e-7 * scale + 1e-10
    # the box is not wider than needed: it excludes pixels far outside the support
    xs, ys = oracle.support_pixels(P, n, 1, cams[0], 2, margin=3.0)
    pr = oracle.project(P, n, 1, cams[0])
    a, _, c = pr["cov"][2]
    assert xs.max() - xs.min() <= 2 * math.sqrt(a) + 8 and ys.max() - ys.min() <= 2 * math.sqrt(c) + 8
    assert ys.max() - ys.min() > xs.max() - xs.min() + 4     # tall splat: tall box


# --------------------------------------------------------------------------
# rule B1 / rule D (binning definition)
# --------------------------------------------------------------------------

def test_rule_exp_within_two_ulp():
    xs = np.concatenate([np.linspace(-80, 80, 4001), np.random.default_rng(0).normal(-5, 1, 2000)]).astype(np.float32)
    for x in xs:
        e = np.float32(oracle.rule_exp(float(x)))
        r = np.float32(np.exp(np.float64(x)))
        assert abs(int(e.view(np.int32)) - int(r.view(np.int32))) <= 2, x


def test_rule_d_key_orders_by_camera_depth():
    sc = scenes.config_scene(1, n=2000)
    cam = sc.cameras[0]
    _, keys, _ = oracle.rule_rects(sc.planes, sc.n, sc.n_lobes, cam)
    depth = oracle.project(sc.planes, sc.n, sc.n_lobes, cam)["depth"]
    kf = keys.view(np.float32)
    assert np.abs(kf - depth).max() < 1e-5 * np.abs(depth).max()
    sep = np.argsort(depth)
    d = depth[sep]
    ok = np.diff(d) > 1e-5
    assert np.all(np.diff(kf[sep].astype(np.float64))[ok] > 0)


@pytest.mark.parametrize("cfg,n", [(1, 4096), (2, 3000), (3, 3000)])
def test_rule_b1_rect_is_conservative_and_tight(cfg, n):
    """Every pixel whose centre has FP64 r^2 < 1 lies in a tile of the
    primitive's rule-B1 rectangle; the rectangle is at most one tile wider on
    each side than the tiles those pixels occupy."""
    sc = scenes.config_scene(cfg, n=n)
    cam = sc.cameras[0]
    pr = oracle.project(sc.planes, sc.n, sc.n_lobes, cam)
    rects, _, binned = oracle.rule_rects(sc.planes, sc.n, sc.n_lobes, cam)
    checked = 0
    for i in range(sc.n):
        if not pr["valid"][i]:
            assert not binned[i]
            continue
        a, b, c = pr["cov"][i]
        mx, my = pr["mu2"][i]
        ex, ey = math.sqrt(a), math.sqrt(c)
        x0, x1 = max(0, int(math.floor(mx - ex - 1))), min(cam.width - 1, int(math.ceil(mx + ex + 1)))
        y0, y1 = max(0, int(math.floor(my - ey - 1))), min(cam.height - 1, int(math.ceil(my + ey + 1)))
        if x0 > x1 or y0 > y1:
            continue
        ys, xs = np.mgrid[y0:y1 + 1, x0:x1 + 1]
        dx, dy = xs + 0.5 - mx, ys + 0.5 - my
        A, B, Cc = pr["conic"][i]
        inside = (A * dx * dx + 2 * B * dx * dy + Cc * dy * dy) < 1.0
        if not inside.any():
            continue
        checked += 1
        assert binned[i], i
        tx, ty = xs[inside] // 16, ys[inside] // 16
        r = rects[i]
        assert r[0] <= tx.min() and tx.max() <= r[1] and r[2] <= ty.min() and ty.max() <= r[3], i
        assert r[0] >= tx.min() - 1 and r[1] <= tx.max() + 1 and r[2] >= ty.min() - 1 and r[3] <= ty.max() + 1
    assert checked > n // 4


def _min_r2_on_rect(Q, mx, my, x0, x1, y0, y1):
    """Minimum of the convex r^2 = d^T Q d (d = p - mu) over the rectangle
    [x0, x1] x [y0, y1] (FP64, closed form: the interior minimum if the centre
    is inside, else the least of the four edge minima)."""
    A, B, C = Q
    if x0 <= mx <= x1 and y0 <= my <= y1:
        return 0.0
    best = np.inf
    for yy in (y0, y1):          # horizontal edges: minimise over x
        dy = yy - my
        dx = float(np.clip(-B * dy / A, x0 - mx, x1 - mx))
        best = min(best, A * dx * dx + 2 * B * dx * dy + C * dy * dy)
    for xx in (x0, x1):          # vertical edges: minimise over y
        dx = xx - mx
        dy = float(np.clip(-B * dx / C, y0 - my, y1 - my))
        best = min(best, A * dx * dx + 2 * B * dx * dy + C * dy * dy)
    return best


def _check_b2(planes, n, n_lobes, cam, tw, th, blur=0.0, stride=1):
    """Rule B2 against FP64: every pixel with r^2 < 1 lies in a kept tile
    (conservative), and in rectangles of 2 x 2 to 32 tiles (the rule's domain)
    every kept tile's rectangle of pixel centres comes within r^2 < 1.002 of
    the support once widened by 1/32 pixel (tight: only the rule's inflation
    and padding separate it from the ellipse).  Returns (primitives checked,
    tiles kept, tiles of the rectangles)."""
    pr = oracle.project(planes, n, n_lobes, cam, blur_eps=blur)
    rects, _, binned, masks = oracle.rule_rects(planes, n, n_lobes, cam, blur, tw, th, with_tiles=True)
    checked = kept_total = rect_total = 0
    for i in range(0, n, stride):
        if not binned[i]:
            continue
        a, b, c = pr["cov"][i]
        mx, my = pr["mu2"][i]
        Q = pr["conic"][i]
        r = rects[i]
        w, h = r[1] - r[0] + 1, r[3] - r[2] + 1
        full = w * h > 32
        kept = set()
        for k in range(w * h):
            if full or (int(masks[i]) >> k) & 1:
                kept.add((r[0] + k % w, r[2] + k // w))
        kept_total += len(kept)
        rect_total += w * h
        ex, ey = math.sqrt(a), math.sqrt(c)
        x0, x1 = max(0, int(math.floor(mx - ex - 1))), min(cam.width - 1, int(math.ceil(mx + ex + 1)))
        y0, y1 = max(0, int(math.floor(my - ey - 1))), min(cam.height - 1, int(math.ceil(my + ey + 1)))
        if x0 <= x1 and y0 <= y1:
            ys, xs = np.mgrid[y0:y1 + 1, x0:x1 + 1]
            dx, dy = xs + 0.5 - mx, ys + 0.5 - my
            inside = (Q[0] * dx * dx + 2 * Q[1] * dx * dy + Q[2] * dy * dy) < 1.0
            need = set(zip((xs[inside] // tw).tolist(), (ys[inside] // th).tolist()))
            assert need <= kept, (i, need - kept)
            checked += bool(need)
        if not full and w >= 2 and h >= 2:      # the rule's domain (others keep the rectangle)
            e = 1.0 / 32
            for (tx, ty) in kept:
                X0, X1 = tx * tw + 0.5 - e, min(tx * tw + tw - 1, cam.width - 1) + 0.5 + e
                Y0, Y1 = ty * th + 0.5 - e, min(ty * th + th - 1, cam.height - 1) + 0.5 + e
                assert _min_r2_on_rect(Q, mx, my, X0, X1, Y0, Y1) < 1.002, (i, tx, ty)
    return checked, kept_total, rect_total


@pytest.mark.parametrize("cfg,n,tile", [(1, 4096, (16, 16)), (2, 20_000, (16, 8)), (3, 20_000, (16, 8)),
                                        (3, 20_000, (8, 8)), (3, 20_000, (32, 16))])
def test_rule_b2_tiles_conservative_and_tight(cfg, n, tile):
    """Rule B2 keeps exactly the tiles of the rule-B1 rectangle the support
    ellipse reaches (Sec. 3.1, Eq. 2: zero contribution outside r^2 < 1):
    none that a pixel with FP64 r^2 < 1 needs is dropped, and each kept one
    lies within the rule's inflation of the ellipse.  On the sheet scenes it
    drops a few percent of the rectangle's tiles."""
    sc = scenes.config_scene(cfg, n=n)
    checked, kept, total = _check_b2(sc.planes, sc.n, sc.n_lobes, sc.cameras[0], *tile)
    assert checked > n // 8
    if cfg == 3:
        assert kept < 0.985 * total


def test_rule_b2_thin_rotated_huge_and_blurred_splats():
    """Edge cases of rule B2 against FP64: thin sheets at many in-plane
    angles and tilts (the x-range of a band comes from the rightmost or
    leftmost point, or from the band's ends, on either side), splats larger
    than the image, splats cut by every image edge, and a 2D blur."""
    rng = np.random.default_rng(8)
    prims = []
    for k in range(120):
        ang = rng.uniform(0, 2 * math.pi)
        tilt = rng.uniform(-1.4, 1.4)
        q = helpers_quat(ang, tilt)
        s = (rng.uniform(0.05, 0.4), rng.uniform(0.003, 0.02), rng.uniform(0.05, 0.4))
        mu = (rng.uniform(-1.4, 1.4), rng.uniform(-1.0, 1.0), rng.uniform(3.0, 6.0))
        prims.append(prim(mu=mu, scale=s, quat=q, opacity=0.5))
    prims.append(prim(mu=(0.0, 0.0, 1.0), scale=(2.0, 0.3, 0.2), opacity=0.5))     # wider than the image
    prims.append(prim(mu=(0.3, 0.2, 2.0), scale=(0.01, 1.5, 0.01), opacity=0.5))   # taller than the image
    P = planes_of(prims)
    n = len(prims)
    cam = scenes.pinhole(np.eye(3, dtype=np.float32), np.zeros(3, np.float32), 173, 131)
    for tw, th in ((16, 16), (16, 8), (8, 8)):
        for blur in (0.0, 0.3):
            checked, kept, total = _check_b2(P, n, 0, cam, tw, th, blur=blur)
            assert checked > n // 2 and kept < total


def helpers_quat(ang, tilt):
    """Quaternion of a rotation by `tilt` about x followed by `ang` about z."""
    qa = axis_angle_quat((0.0, 0.0, 1.0), ang)
    qt = axis_angle_quat((1.0, 0.0, 0.0), tilt)
    w1, x1, y1, z1 = qa
    w2, x2, y2, z2 = qt
    return (w1 * w2 - x1 * x2 - y1 * y2 - z1 * z2, w1 * x2 + x1 * w2 + y1 * z2 - z1 * y2,
            w1 * y2 - x1 * z2 + y1 * w2 + z1 * x2, w1 * z2 + x1 * y2 - y1 * x2 + z1 * w2)


def test_bin_pairs_sorted_and_complete():
    sc = scenes.config_scene(1, n=1500)
    tiles, recs, ranges = oracle.bin_pairs(sc.planes, sc.n, sc.n_lobes, sc.cameras)
    assert np.all(np.diff(tiles.astype(np.int64)) >= 0)
    rects, keys, binned, masks = oracle.rule_rects(sc.planes, sc.n, sc.n_lobes, sc.cameras[0], with_tiles=True)
    area = (rects[:, 1] - rects[:, 0] + 1) * (rects[:, 3] - rects[:, 2] + 1)
    bits = np.array([bin(int(m)).count("1") for m in masks])
    cnt = np.where(area > 32, area, bits)[binned > 0].sum()
    assert len(tiles) == cnt
    for g in range(len(ranges) - 1):
        seg = recs[ranges[g]:ranges[g + 1]]
        k = keys[seg]
        assert np.all((np.diff(k.astype(np.int64)) > 0) | ((np.diff(k.astype(np.int64)) == 0) & (np.diff(seg.astype(np.int64)) > 0)))


# --------------------------------------------------------------------------
# the paper's printed constants
# --------------------------------------------------------------------------

def test_paper_constants_golden():
    with open(os.path.join(GOLDEN, "paper_constants.json")) as fh:
        g = json.load(fh)
    assert scenes.n_planes(0) - 3 == g["geometry_floats_per_primitive"]
    assert 3 + 6 * 2 == g["sb2_feature_dim"]
    sh3 = g["sh_degree3_feature_dim"]
    assert abs((3 + 6 * 2) / sh3 - g["sb_vs_sh_param_fraction"]) < 0.01
    dbs, gs = scenes.n_planes(2), 3 + 3 + 4 + 1 + sh3
    assert abs(dbs / gs - g["dbs_vs_3dgs_param_fraction"]) < 0.01
    # c = 4: int_0^1 (1-x)^4 dx = 1/5 vs int_0^1 e^{-9x/2} dx (the paper's approximation)
    assert abs(1.0 / (g["beta_c"] + 1) - g["beta_c_integral"]) < 1e-12
    assert abs((1 - math.exp(-4.5)) / 4.5 - g["gaussian_integral"]) < 1e-4
    assert abs(g["noise_b_prime"] - math.log(25.0)) < 1e-12


# --------------------------------------------------------------------------
# geometry decomposition (Sec. 4.3): render the primitives with b in a range
# --------------------------------------------------------------------------

def test_geometry_decomposition_equals_removing_primitives():
    """Masking by b_lo <= b < b_hi renders exactly the scene without the other
    primitives, and bins exactly the kept ones."""
    sc = scenes.config_scene(1, n=600, seed=5)
    cam = scenes.pinhole(*scenes.look_at((0.0, 0.0, -3.0)), 64, 48)
    b = sc.planes[11, :sc.n]
    thr = float(np.float32(b.mean()))
    for lo, hi in ((-np.inf, thr), (thr, np.inf)):
        keep = np.nonzero((b >= np.float32(lo)) & (b < np.float32(hi)))[0]
        sub = np.ascontiguousarray(sc.planes[:, keep])
        full = oracle.render_full(sc.planes, sc.n, sc.n_lobes, cam, b_lo=lo, b_hi=hi)
        only = oracle.render_full(sub, len(keep), sc.n_lobes, cam)
        assert np.array_equal(full[0], only[0]) and np.array_equal(full[1], only[1])
        _, recs, _ = oracle.bin_pairs(sc.planes, sc.n, sc.n_lobes, [cam], b_lo=lo, b_hi=hi)
        assert set(np.unique(recs)) <= set(keep)
        _, recs_sub, _ = oracle.bin_pairs(sub, len(keep), sc.n_lobes, [cam])
        assert len(recs) == len(recs_sub)
