"""FP64 oracle of the optimiser step around the rasterizer (test
infrastructure: only tests/, __graft_entry__.smoke() and bench.py's CPU legs
may use it).

One training step after the rasterizer's backward (Sec. 3.4, "Kernel-Agnostic
Markov Chain Monte Carlo", Optimization paragraph and the composite loss;
hyperparameters from the appendix "Hyperparameters"):

  * regularisers of the composite loss: lambda_o * sum_i |o_i| and
    lambda_Sigma * sum_i sum_j |sqrt(eig_j(Sigma_i))|.  With Sigma = R S S^T R^T
    the square roots of the eigenvalues are the scales s_j = exp(log-scale_j),
    and o = sigmoid(logit) > 0, so the gradients w.r.t. the raw parameters
    are lambda_o o (1 - o) and lambda_Sigma s_j;
  * Adam on every raw parameter (first and second moments, bias-corrected),
    one learning rate per parameter group;
  * the position noise mu <- mu + lambda_eps * eps with
    eps = lr_mu * B(o; b') * Sigma eta, B(o; b') = (1 - o)^(4 e^b') the Beta
    kernel of Eq. eq:beta, b' = ln 25, and eta ~ N(0, I_3) supplied by the
    caller (the sampled noise).

Readings (the paper is silent): the optimiser is Adam (beta1 0.9, beta2
0.999, eps 1e-15), "Sigma_eta" is the primitive's 3D covariance applied to a
standard normal sample, and the noise, like the gradient step, is computed
from the parameters as they were before the step.
"""
from __future__ import annotations

import math

import numpy as np

P_MEAN, P_LOGSCALE, P_QUAT, P_OPACITY, P_B, P_C0, P_LOBES = 0, 3, 6, 10, 11, 12, 15
LOBE_STRIDE = 6

# parameter groups and their learning rates (appendix "Hyperparameters")
GROUPS = ("mean", "log_scale", "quat", "opacity", "b", "c0", "lobe_dir", "lobe_b", "lobe_color")
PAPER_LR = {"mean": 1.6e-4, "log_scale": 5e-3, "quat": 1e-3, "opacity": 5e-2, "b": 1e-3, "c0": 2.5e-3,
            "lobe_dir": 2.5e-3, "lobe_b": 2.5e-3, "lobe_color": 2.5e-3}


def plane_groups(n_lobes: int) -> list[int]:
    """Group index (into GROUPS) of every parameter plane."""
    g = [0, 0, 0, 1, 1, 1, 2, 2, 2, 2, 3, 4, 5, 5, 5]
    for _ in range(n_lobes):
        g += [6, 6, 7, 8, 8, 8]
    return g


def beta_kernel(x, b):
    """B(x; b) = (1 - x)^(4 e^b), Eq. eq:beta."""
    return (1.0 - x) ** (4.0 * math.exp(b))


def rotation(q):
    """Rotation matrices (n,3,3) of quaternions q = (w, x, y, z) (n,4), normalised here."""
    q = q / np.linalg.norm(q, axis=1, keepdims=True)
    w, x, y, z = q.T
    return np.stack([
        np.stack([1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)], -1),
        np.stack([2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)], -1),
        np.stack([2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)], -1)], 1)


def regularisers(planes, n, lambda_o, lambda_sigma):
    """(lambda_o sum o, lambda_Sigma sum_j s_j) of the first n primitives."""
    p = np.asarray(planes, np.float64)[:, :n]
    o = 1.0 / (1.0 + np.exp(-p[P_OPACITY]))
    s = np.exp(p[P_LOGSCALE:P_LOGSCALE + 3])
    return lambda_o * o.sum(), lambda_sigma * s.sum()


def regulariser_grad(planes, n, lambda_o, lambda_sigma):
    """Gradient planes of regularisers() w.r.t. the raw parameters."""
    p = np.asarray(planes, np.float64)
    g = np.zeros_like(p)
    o = 1.0 / (1.0 + np.exp(-p[P_OPACITY, :n]))
    g[P_OPACITY, :n] = lambda_o * o * (1.0 - o)
    g[P_LOGSCALE:P_LOGSCALE + 3, :n] = lambda_sigma * np.exp(p[P_LOGSCALE:P_LOGSCALE + 3, :n])
    return g


def adam_step(planes, grad, m, v, eta, n, n_lobes, lr, step, beta1=0.9, beta2=0.999, eps=1e-15,
              lambda_o=0.01, lambda_sigma=0.01, lambda_eps=5e4, noise_b=math.log(25.0)):
    """One optimiser step on the first n columns of the SoA planes.

    planes, grad, m, v: (15 + 6 M, pitch) arrays; eta: (3, pitch) standard
    normal samples; lr: dict group -> learning rate (mean: the current
    position rate lambda_lr).  Returns new (planes, m, v) as float64 arrays
    and the two regulariser values."""
    P = np.array(planes, np.float64)
    G = np.array(grad, np.float64)
    M = np.array(m, np.float64)
    V = np.array(v, np.float64)
    E = np.asarray(eta, np.float64)
    cols = slice(0, n)
    o = 1.0 / (1.0 + np.exp(-P[P_OPACITY, cols]))
    s = np.exp(P[P_LOGSCALE:P_LOGSCALE + 3, cols])
    R = rotation(P[P_QUAT:P_QUAT + 4, cols].T)
    reg = regularisers(P, n, lambda_o, lambda_sigma)
    # regulariser gradients
    G += regulariser_grad(P, n, lambda_o, lambda_sigma)
    # position noise from the pre-step parameters: Sigma eta, Sigma = R diag(s^2) R^T
    cov = np.einsum("nij,jn,nkj->nik", R, s * s, R)
    sig_eta = np.einsum("nik,kn->in", cov, E[:, cols])
    noise = lambda_eps * lr["mean"] * beta_kernel(o, noise_b) * sig_eta
    # Adam
    groups = plane_groups(n_lobes)
    c1 = 1.0 - beta1 ** step
    c2 = 1.0 - beta2 ** step
    for k in range(P.shape[0]):
        g = G[k, cols]
        M[k, cols] = beta1 * M[k, cols] + (1.0 - beta1) * g
        V[k, cols] = beta2 * V[k, cols] + (1.0 - beta2) * g * g
        mh = M[k, cols] / c1
        vh = V[k, cols] / c2
        P[k, cols] -= lr[GROUPS[groups[k]]] * mh / (np.sqrt(vh) + eps)
    P[P_MEAN:P_MEAN + 3, cols] += noise
    return P, M, V, reg


# ---------------------------------------------------------------------------
# Relocation of dead primitives (Sec. 3.4 "Densification", Eq. eq:densify):
# a primitive whose opacity is below min_opacity is dead; it is respawned as
# a copy of a live primitive drawn by multinomial sampling with probabilities
# proportional to opacity (with replacement, one draw per dead primitive, in
# index order); a live primitive that ends up with N copies in total
# (itself included) gets o' = 1 - (1 - o)^(1/N) on all of them, its other
# parameters unchanged (opacity-only adjustment).  The copies' optimiser
# moments are reset to zero.
#
# Decisions are integers: dead = rule_opacity(logit) < min_opacity with the
# fixed fp32 rule, weight = floor(rule_opacity * 2^24) for live primitives,
# inclusive cumulative sum W (64-bit integers); the caller's 32-bit random
# word r picks t = floor(r W_total / 2^32) and the source is the first i with
# W_i > t.  The new opacities are FP64.
# ---------------------------------------------------------------------------

def relocate(planes, m, v, rnd, n, min_opacity):
    """Returns new (planes, m, v) (float64), the source index of every
    primitive (-1: kept) and the number relocated."""
    from . import rule_opacity
    P = np.array(planes, np.float64)
    Mo = np.array(m, np.float64)
    Vo = np.array(v, np.float64)
    src = np.full(n, -1, np.int64)
    if n == 0:
        return P, Mo, Vo, src, 0
    o32 = rule_opacity(np.asarray(planes, np.float32)[P_OPACITY, :n])
    dead = o32 < np.float32(min_opacity)
    w = np.where(dead, 0, (o32 * np.float32(16777216.0)).astype(np.uint64)).astype(np.uint64)
    cdf = np.cumsum(w, dtype=np.uint64)
    total = int(cdf[-1])
    if total == 0:
        return P, Mo, Vo, src, 0
    dead_idx = np.nonzero(dead)[0]
    for d in dead_idx:
        t = (int(rnd[d]) * total) >> 32
        src[d] = int(np.searchsorted(cdf, np.uint64(t), side="right"))
    copies = np.bincount(src[dead_idx], minlength=n) if len(dead_idx) else np.zeros(n, np.int64)
    for s in np.nonzero(copies)[0]:
        N = copies[s] + 1
        o = 1.0 / (1.0 + math.exp(-P[P_OPACITY, s]))
        o_new = -math.expm1(math.log1p(-o) / N)
        P[P_OPACITY, s] = math.log(o_new) - math.log1p(-o_new)
    for d in dead_idx:
        P[:, d] = P[:, src[d]]
        Mo[:, d] = 0.0
        Vo[:, d] = 0.0
    return P, Mo, Vo, src, len(dead_idx)
