"""FP64 oracle of the image loss with the DSSIM term (test infrastructure:
only tests/, __graft_entry__.smoke() and bench.py's CPU legs may use it).

The composite loss of Sec. 3.4 weights the pixel-wise L1 term by
(1 - lambda_SSIM) and the SSIM term by lambda_SSIM (0.2 in the appendix
"Hyperparameters").  Per view v with colour x and target y (3 x H x W):

    loss_v = (1 - lambda) mean|x - y| + lambda (1 - mean SSIM(x, y)),

SSIM per pixel and channel from Gaussian-weighted local statistics:
    mu_x = G * x,  sigma_x^2 = G * x^2 - mu_x^2,  sigma_xy = G * (x y) - mu_x mu_y,
    SSIM = (2 mu_x mu_y + C1)(2 sigma_xy + C2) / ((mu_x^2 + mu_y^2 + C1)(sigma_x^2 + sigma_y^2 + C2)).

Readings (the paper names the term only): an 11-tap Gaussian window with
sigma 1.5 applied separably, zero padding outside the image ("same" size),
C1 = 0.01^2 and C2 = 0.03^2 for a dynamic range of 1, the SSIM term as
1 - SSIM, means over the view's three channels and pixels.

grad() is the analytic gradient w.r.t. x, written out here from the chain
rule through (mu_x, G * x^2, G * x y); the tests pin it against finite
differences of loss().
"""
from __future__ import annotations

import numpy as np

WIN = 11
SIGMA = 1.5
C1 = 0.01 ** 2
C2 = 0.03 ** 2


def window() -> np.ndarray:
    """The normalised 1D Gaussian taps (11)."""
    k = np.arange(WIN, dtype=np.float64) - WIN // 2
    g = np.exp(-k * k / (2.0 * SIGMA * SIGMA))
    return g / g.sum()


def blur(img: np.ndarray) -> np.ndarray:
    """Separable Gaussian filter of an (H, W) image, zero padding, same size."""
    g = window()
    r = WIN // 2
    H, W = img.shape
    p = np.pad(np.asarray(img, np.float64), ((0, 0), (r, r)))
    h = sum(g[k] * p[:, k:k + W] for k in range(WIN))
    p = np.pad(h, ((r, r), (0, 0)))
    return sum(g[k] * p[k:k + H, :] for k in range(WIN))


def _stats(x, y):
    mx, my = blur(x), blur(y)
    sxx = blur(x * x) - mx * mx
    syy = blur(y * y) - my * my
    sxy = blur(x * y) - mx * my
    return mx, my, sxx, syy, sxy


def ssim_map(x: np.ndarray, y: np.ndarray) -> np.ndarray:
    """Per-pixel SSIM of two (H, W) channels."""
    mx, my, sxx, syy, sxy = _stats(np.asarray(x, np.float64), np.asarray(y, np.float64))
    return ((2 * mx * my + C1) * (2 * sxy + C2)) / ((mx * mx + my * my + C1) * (sxx + syy + C2))


def loss(color: np.ndarray, target: np.ndarray, lam: float = 0.2) -> float:
    """loss_v of one view; color, target (3, H, W)."""
    x = np.asarray(color, np.float64)
    y = np.asarray(target, np.float64)
    l1 = np.abs(x - y).mean()
    s = np.mean([ssim_map(x[c], y[c]).mean() for c in range(x.shape[0])])
    return (1.0 - lam) * l1 + lam * (1.0 - s)


def grad(color: np.ndarray, target: np.ndarray, lam: float = 0.2) -> np.ndarray:
    """d loss_v / d color, (3, H, W).  The L1 part takes sign(0) = 0."""
    x = np.asarray(color, np.float64)
    y = np.asarray(target, np.float64)
    N = x.size
    out = (1.0 - lam) * np.sign(x - y) / N
    for c in range(x.shape[0]):
        xc, yc = x[c], y[c]
        mx, my, sxx, syy, sxy = _stats(xc, yc)
        A1, A2 = 2 * mx * my + C1, 2 * sxy + C2
        B1, B2 = mx * mx + my * my + C1, sxx + syy + C2
        S = A1 * A2 / (B1 * B2)
        d = 1.0 / (B1 * B2)
        # S as a function of (mu_x, G * x^2, G * x y) at each pixel p:
        #   dS/dE[x^2] = dS/dsigma_x^2 = -S / B2,  dS/dE[xy] = dS/dsigma_xy = 2 A1 d,
        #   dS/dmu_x = 2 mu_y A2 d - 2 mu_x S / B1 - 2 mu_x dS/dsigma_x^2 - mu_y dS/dsigma_xy
        d_e2 = -S / B2
        d_xy = 2 * A1 * d
        a = 2 * my * A2 * d - 2 * mx * S / B1 - 2 * mx * d_e2 - my * d_xy
        # dS_p/dx_q = G_pq (a_p + 2 x_q d_e2_p + y_q d_xy_p); the window is symmetric
        dS = blur(a) + 2 * xc * blur(d_e2) + yc * blur(d_xy)
        out[c] -= lam * dS / N
    return out
