"""Pins of the FP64 optimiser-step oracle (Sec. 3.4 Optimization paragraph,
the composite loss, appendix Hyperparameters) against closed forms: Adam with
a constant or alternating gradient, the regulariser gradients against finite
differences, and the position noise for primitives whose covariance and
opacity make Sigma eta and B(o; b') known exactly."""
import math

import numpy as np
import pytest

from oracle import optim

M_LOBES = 1
NP = 15 + 6 * M_LOBES
ZERO = dict(lambda_o=0.0, lambda_sigma=0.0, lambda_eps=0.0)


def planes_for(n, rng):
    p = rng.normal(size=(NP, n))
    p[optim.P_QUAT:optim.P_QUAT + 4] += np.array([[2.0], [0.0], [0.0], [0.0]])
    return p


def lr_all(x=1e-3):
    return {g: x for g in optim.GROUPS}


def test_first_step_is_lr_times_sign():
    rng = np.random.default_rng(1)
    p0, g = planes_for(7, rng), rng.normal(size=(NP, 7))
    z = np.zeros_like(p0)
    lr = {k: 10.0 ** -(i + 1) for i, k in enumerate(optim.GROUPS)}
    p1, m1, v1, _ = optim.adam_step(p0, g, z, z, np.zeros((3, 7)), 7, M_LOBES, lr, 1, **ZERO)
    groups = optim.plane_groups(M_LOBES)
    rates = np.array([lr[optim.GROUPS[groups[k]]] for k in range(NP)])[:, None]
    # g / (|g| + eps) is sign(g) to eps / |g|
    assert np.allclose(p1, p0 - rates * np.sign(g), rtol=0, atol=1e-12)
    assert np.allclose(m1, 0.1 * g, rtol=1e-15) and np.allclose(v1, 0.001 * g * g, rtol=1e-12)


def test_constant_gradient_moves_lr_per_step():
    rng = np.random.default_rng(2)
    p, g = planes_for(5, rng), rng.normal(size=(NP, 5))
    m = v = np.zeros_like(p)
    p0 = p.copy()
    for t in range(1, 6):
        p, m, v, _ = optim.adam_step(p, g, m, v, np.zeros((3, 5)), 5, M_LOBES, lr_all(), t, **ZERO)
    assert np.allclose(p, p0 - 5 * 1e-3 * np.sign(g), rtol=0, atol=1e-12)


def test_alternating_gradient_closed_form():
    # g then -g: m2 = -0.01 g, bias-corrected -g/19; v2 bias-corrected = g^2
    g = np.full((NP, 3), 0.7)
    p0 = np.zeros((NP, 3))
    p0[optim.P_QUAT] = 1.0
    z = np.zeros_like(p0)
    p1, m1, v1, _ = optim.adam_step(p0, g, z, z, np.zeros((3, 3)), 3, M_LOBES, lr_all(), 1, **ZERO)
    p2, _, _, _ = optim.adam_step(p1, -g, m1, v1, np.zeros((3, 3)), 3, M_LOBES, lr_all(), 2, **ZERO)
    assert np.allclose(p2, p0 - 1e-3 + 1e-3 / 19.0, rtol=0, atol=1e-14)


def test_regulariser_gradient_matches_finite_differences():
    rng = np.random.default_rng(3)
    p = planes_for(4, rng)
    g = optim.regulariser_grad(p, 4, 0.01, 0.02)
    h = 1e-6
    for k in [optim.P_OPACITY, optim.P_LOGSCALE, optim.P_LOGSCALE + 1, optim.P_LOGSCALE + 2]:
        for i in range(4):
            a, b = p.copy(), p.copy()
            a[k, i] += h
            b[k, i] -= h
            fd = (sum(optim.regularisers(a, 4, 0.01, 0.02)) - sum(optim.regularisers(b, 4, 0.01, 0.02))) / (2 * h)
            assert g[k, i] == pytest.approx(fd, rel=1e-7, abs=1e-12)
    # the step adds it to the loss gradient: first moments after one step
    z = np.zeros_like(p)
    _, m1, _, _ = optim.adam_step(p, z, z, z, np.zeros((3, 4)), 4, M_LOBES, lr_all(), 1,
                                  lambda_o=0.01, lambda_sigma=0.02, lambda_eps=0.0)
    assert np.allclose(m1, 0.1 * g, rtol=1e-14, atol=0)


def test_regulariser_values():
    p = np.zeros((NP, 2))
    p[optim.P_OPACITY] = [0.0, math.log(3.0)]             # o = 1/2, 3/4
    p[optim.P_LOGSCALE:optim.P_LOGSCALE + 3] = np.log([[1.0, 2.0], [3.0, 4.0], [5.0, 6.0]])
    ro, rs = optim.regularisers(p, 2, 0.01, 0.1)
    assert ro == pytest.approx(0.01 * 1.25, rel=1e-14)
    assert rs == pytest.approx(0.1 * 21.0, rel=1e-14)


def _noise_case(logit, quat, log_scale, eta, lam=5e4, lr_mu=1.6e-4):
    p = np.zeros((NP, 1))
    p[optim.P_OPACITY] = logit
    p[optim.P_QUAT:optim.P_QUAT + 4, 0] = quat
    p[optim.P_LOGSCALE:optim.P_LOGSCALE + 3, 0] = log_scale
    z = np.zeros_like(p)
    lr = lr_all(0.0)
    lr["mean"] = lr_mu
    p1, _, _, _ = optim.adam_step(p, z, z, z, np.array(eta, float).reshape(3, 1), 1, M_LOBES, lr, 1,
                                  lambda_o=0.0, lambda_sigma=0.0, lambda_eps=lam)
    return p1[:3, 0] - p[:3, 0]


def test_noise_axis_aligned_transparent_primitive():
    # o ~ 4e-18: B(o; ln 25) = 1; identity rotation: Sigma eta = s^2 * eta
    d = _noise_case(-40.0, [1, 0, 0, 0], np.log([2.0, 3.0, 0.5]), [1.0, 1.0, 1.0])
    assert np.allclose(d, 5e4 * 1.6e-4 * np.array([4.0, 9.0, 0.25]), rtol=1e-12)


def test_noise_follows_rotation_and_ignores_quaternion_norm():
    # 90 degrees about z, quaternion scaled by 2: the primitive's x axis is world y
    c = math.cos(math.pi / 4)
    d = _noise_case(-40.0, [2 * c, 0, 0, 2 * c], np.log([2.0, 3.0, 0.5]), [0.0, 1.0, 0.0])
    assert np.allclose(d, 5e4 * 1.6e-4 * np.array([0.0, 4.0, 0.0]), rtol=1e-12, atol=1e-12)


def test_noise_vanishes_for_opaque_primitives():
    d = _noise_case(40.0, [1, 0, 0, 0], np.log([2.0, 3.0, 0.5]), [1.0, 1.0, 1.0])
    assert np.all(d == 0.0)


def test_noise_scale_is_the_beta_kernel_at_b_ln25():
    # o = 1/2: B = (1/2)^(4 * 25) = 2^-100
    d = _noise_case(0.0, [1, 0, 0, 0], [0.0, 0.0, 0.0], [1.0, 0.0, 0.0])
    assert d[0] == pytest.approx(5e4 * 1.6e-4 * 2.0 ** -100, rel=1e-12)
    assert optim.beta_kernel(0.25, math.log(25.0)) == pytest.approx(0.75 ** 100, rel=1e-14)


# ---------------------------------------------------------------------------
# relocation (Sec. 3.4 Densification, Eq. eq:densify)
# ---------------------------------------------------------------------------

def _reloc_planes(logits):
    n = len(logits)
    p = np.zeros((NP, n))
    p[optim.P_OPACITY] = logits
    p[:3] = np.arange(3 * n).reshape(3, n)        # distinct positions identify copies
    p[optim.P_QUAT] = 1.0
    return p


def test_relocation_preserves_the_combined_opacity():
    # one live primitive (o = 0.3), two dead ones: three copies of o' with
    # 1 - (1 - o')^3 = o (Eq. eq:densify at the centre, f = 1)
    logit = math.log(0.3 / 0.7)
    p = _reloc_planes([logit, -20.0, -20.0])
    m = np.ones_like(p)
    P, Mo, Vo, src, k = optim.relocate(p, m, m, np.array([1, 2**31, 2**32 - 1], np.uint64), 3, 0.005)
    assert k == 2 and list(src) == [-1, 0, 0]
    o_new = 1.0 / (1.0 + np.exp(-P[optim.P_OPACITY]))
    assert np.allclose(o_new, o_new[0]) and 1.0 - (1.0 - o_new[0]) ** 3 == pytest.approx(0.3, rel=1e-12)
    assert np.all(P[:3, 1] == p[:3, 0]) and np.all(P[:3, 2] == p[:3, 0])     # copies of the source
    assert np.all(Mo[:, 1:] == 0) and np.all(Mo[:, 0] == 1) and np.all(Vo[:, 1:] == 0)


def test_relocation_small_opacity_is_o_over_n():
    # Taylor reading of the paper: o' = 1 - (1 - o)^(1/N) ~ o / N for small o
    o = 0.01
    p = _reloc_planes([math.log(o / (1 - o))] + [-30.0] * 4)
    P, _, _, src, k = optim.relocate(p, np.zeros_like(p), np.zeros_like(p), np.zeros(5, np.uint64), 5, 0.005)
    assert k == 4 and np.all(src[1:] == 0)
    o_new = 1.0 / (1.0 + math.exp(-P[optim.P_OPACITY, 0]))
    assert o_new == pytest.approx(o / 5, rel=o)                 # error O(o)
    assert o_new == pytest.approx(1 - (1 - o) ** 0.2, rel=1e-12)


def test_relocation_samples_in_proportion_to_opacity():
    # live opacities 0.1 / 0.3 / 0.6; random words spread uniformly over
    # [0, 2^32): the draws are non-decreasing in the word and hit each source
    # in proportion to its opacity
    lo = [math.log(x / (1 - x)) for x in (0.1, 0.3, 0.6)]
    nd = 2000
    p = _reloc_planes(lo + [-30.0] * nd)
    rnd = (np.arange(nd, dtype=np.uint64) * (2**32 // nd)).astype(np.uint64)
    rr = np.concatenate([np.zeros(3, np.uint64), rnd])
    _, _, _, src, k = optim.relocate(p, np.zeros_like(p), np.zeros_like(p), rr, 3 + nd, 0.005)
    assert k == nd and np.all(np.diff(src[3:]) >= 0)
    frac = np.bincount(src[3:], minlength=3) / nd
    assert np.allclose(frac, [0.1, 0.3, 0.6], atol=1e-3)


def test_relocation_without_dead_or_live_primitives_is_identity():
    p = _reloc_planes([0.0, 1.0, 2.0])
    P, _, _, src, k = optim.relocate(p, np.zeros_like(p), np.zeros_like(p), np.zeros(3, np.uint64), 3, 0.005)
    assert k == 0 and np.all(src == -1) and np.array_equal(P, p)
    p = _reloc_planes([-30.0, -40.0])
    P, _, _, src, k = optim.relocate(p, np.zeros_like(p), np.zeros_like(p), np.zeros(2, np.uint64), 2, 0.005)
    assert k == 0 and np.array_equal(P, p)
