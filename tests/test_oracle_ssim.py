"""Pins of the FP64 DSSIM-loss oracle (Sec. 3.4 composite loss): the window,
the zero-padded separable filter against a direct 2D sum, SSIM's identity,
symmetry and constant-image closed form, and the analytic gradient against
central finite differences."""
import numpy as np
import pytest

from oracle import ssim


def test_window_is_a_normalised_gaussian():
    g = ssim.window()
    assert len(g) == 11 and g.sum() == pytest.approx(1.0, abs=1e-15)
    assert g[5] / g[6] == pytest.approx(np.exp(1.0 / (2 * 1.5 ** 2)), rel=1e-14)
    assert np.allclose(g, g[::-1])


def test_blur_equals_direct_zero_padded_2d_sum():
    rng = np.random.default_rng(0)
    img = rng.normal(size=(9, 14))
    g = ssim.window()
    K = np.outer(g, g)
    ref = np.zeros_like(img)
    for i in range(9):
        for j in range(14):
            for a in range(-5, 6):
                for b in range(-5, 6):
                    if 0 <= i + a < 9 and 0 <= j + b < 14:
                        ref[i, j] += K[a + 5, b + 5] * img[i + a, j + b]
    assert np.allclose(ssim.blur(img), ref, rtol=0, atol=1e-14)


def test_ssim_identity_and_symmetry():
    rng = np.random.default_rng(1)
    x, y = rng.random((20, 23)), rng.random((20, 23))
    assert np.allclose(ssim.ssim_map(x, x), 1.0, rtol=0, atol=1e-12)
    assert np.allclose(ssim.ssim_map(x, y), ssim.ssim_map(y, x), rtol=0, atol=1e-15)
    assert np.all(ssim.ssim_map(x, y) <= 1.0 + 1e-12)
    c = np.stack([x, x, x])
    assert ssim.loss(c, c) == pytest.approx(0.0, abs=1e-12)
    assert np.allclose(ssim.grad(c, c), 0.0, atol=1e-12)


def test_constant_images_interior_closed_form():
    a, b = 0.3, 0.7
    s = ssim.ssim_map(np.full((30, 30), a), np.full((30, 30), b))
    expect = (2 * a * b + ssim.C1) / (a * a + b * b + ssim.C1)    # sigmas vanish
    assert np.allclose(s[5:-5, 5:-5], expect, rtol=1e-12)


@pytest.mark.parametrize("lam", [0.2, 1.0])
def test_gradient_matches_finite_differences(lam):
    rng = np.random.default_rng(2)
    x = rng.random((3, 12, 13))
    y = rng.random((3, 12, 13))
    g = ssim.grad(x, y, lam)
    h = 1e-6
    for (c, i, j) in [(0, 0, 0), (1, 5, 6), (2, 11, 12), (0, 6, 0), (2, 3, 9), (1, 11, 4)]:
        xp, xm = x.copy(), x.copy()
        xp[c, i, j] += h
        xm[c, i, j] -= h
        fd = (ssim.loss(xp, y, lam) - ssim.loss(xm, y, lam)) / (2 * h)
        assert g[c, i, j] == pytest.approx(fd, rel=1e-6, abs=1e-11)
