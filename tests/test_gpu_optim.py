"""The optimiser step (beta_adam_step) against the FP64 oracle (oracle.optim)
element by element, through the C ABI: ragged primitive counts, padding
columns left untouched, opaque and transparent primitives, several steps."""
import ctypes
import math

import numpy as np
import pytest
import torch

from oracle import optim
from paper_2501_18630_gb300 import _lib, scenes
from paper_2501_18630_gb300.optim import BetaAdam
from tests import gpu_common as gc

pytestmark = pytest.mark.gpu

# the ABI carries the hyperparameters as float32: the oracle takes the same
# numbers (1 - 0.999f differs from 1 - 0.999 by 1.3e-5 relative)
F32 = {k: float(np.float32(v)) for k, v in dict(beta1=0.9, beta2=0.999, eps=1e-15, lambda_o=0.01,
                                                  lambda_sigma=0.01, lambda_eps=5e4,
                                                  noise_b=math.log(25.0)).items()}


def _close(gpu, ref, p0):
    """fp32 step against FP64: a few ulp of the value plus 1e-4 of the change."""
    gpu = gpu.astype(np.float64)
    tol = 4 * np.spacing(np.abs(ref).astype(np.float32)).astype(np.float64) + 1e-4 * np.abs(ref - p0) + 1e-30
    return np.abs(gpu - ref) <= tol


@pytest.mark.parametrize("n,n_lobes", [(1, 0), (4097, 3), (20_000, 2)])
def test_adam_step_matches_oracle(n, n_lobes):
    gc.ensure_built()
    rng = np.random.default_rng(n + n_lobes)
    sc = scenes.config_scene(2 if n_lobes == 2 else 3, n=max(n, 8))
    pitch = scenes.round_pitch(n)
    NP = scenes.n_planes(n_lobes)
    p0 = np.zeros((NP, pitch), np.float32)
    p0[:, :n] = sc.planes[:NP, :n] if sc.n_lobes >= n_lobes else rng.normal(size=(NP, n))
    p0[:, n:] = 7.0                                           # padding columns: must stay
    p0[10, :min(n, 3)] = [-40.0, 40.0, 0.0][:min(n, 3)]        # transparent, opaque, half
    g = rng.normal(scale=1e-2, size=(NP, pitch)).astype(np.float32)
    m0 = rng.normal(scale=1e-3, size=(NP, pitch)).astype(np.float32)
    v0 = (rng.normal(scale=1e-3, size=(NP, pitch)) ** 2).astype(np.float32)
    eta = rng.normal(size=(3, pitch)).astype(np.float32)
    lr = dict(optim.PAPER_LR)
    ref_p, ref_m, ref_v, ref_reg = optim.adam_step(p0, g, m0, v0, eta, n, n_lobes, lr, 3, **F32)
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    P, G, Mm, Vv, E = dev(p0), dev(g), dev(m0), dev(v0), dev(eta)
    reg = torch.zeros(2, dtype=torch.float64, device="cuda")
    o = _lib.adam_default_opts(lr)
    o.step = 3
    vp = lambda t: ctypes.c_void_p(t.data_ptr())
    _lib.check("beta_adam_step", _lib.load().beta_adam_step(n, pitch, n_lobes, vp(P), vp(G), vp(Mm), vp(Vv),
                                                            vp(E), ctypes.byref(o), vp(reg), None))
    torch.cuda.synchronize()
    Pg, Mg, Vg = P.cpu().numpy(), Mm.cpu().numpy(), Vv.cpu().numpy()
    assert np.all(Pg[:, n:] == 7.0)
    assert np.all(_close(Pg[:, :n], ref_p[:, :n], p0[:, :n]))
    # m = b1 m0 + (1 - b1) g can cancel: a few ulp of its terms (g with the
    # regularisers' gradient); v has no cancellation
    gt = np.abs(g.astype(np.float64)) + optim.regulariser_grad(p0, n, F32["lambda_o"], F32["lambda_sigma"])
    mag = (0.9 * np.abs(m0) + 0.1 * gt).astype(np.float32)[:, :n]
    assert np.all(np.abs(Mg[:, :n] - ref_m[:, :n]) <= 4 * np.spacing(mag))
    assert np.allclose(Vg[:, :n], ref_v[:, :n], rtol=4e-6, atol=0)
    r = reg.cpu().numpy()
    assert r[0] == pytest.approx(ref_reg[0], rel=1e-5) and r[1] == pytest.approx(ref_reg[1], rel=1e-5)
    if n >= 3:
        # opaque primitive: no noise, the position moves by the Adam step only
        ref0, _, _, _ = optim.adam_step(p0, g, m0, v0, np.zeros_like(eta), n, n_lobes, lr, 3, **F32)
        assert np.all(_close(Pg[:3, 1], ref0[:3, 1], p0[:3, 1]))


def test_adam_wrapper_steps():
    """Five steps through the Python wrapper (bias correction 1 - beta^t for
    t = 1..5, a decaying position rate): each step from the device state
    matches the oracle's step from the same state."""
    gc.ensure_built()
    rng = np.random.default_rng(5)
    n, n_lobes, pitch = 3000, 1, 3008
    NP = scenes.n_planes(n_lobes)
    planes = torch.from_numpy(rng.normal(size=(NP, pitch)).astype(np.float32)).cuda()
    opt = BetaAdam(planes, n, n_lobes)
    for t in range(1, 6):
        p_prev = planes.cpu().numpy().copy()
        m_prev, v_prev = opt.m.cpu().numpy().copy(), opt.v.cpu().numpy().copy()
        g = rng.normal(scale=1e-2, size=(NP, pitch)).astype(np.float32)
        eta = rng.normal(size=(3, pitch)).astype(np.float32)
        lr_mu = 1.6e-4 * 0.99 ** t
        opt.step(planes, torch.from_numpy(g).cuda(), torch.from_numpy(eta).cuda(), lr_mean=lr_mu)
        ref, _, _, _ = optim.adam_step(p_prev, g, m_prev, v_prev, eta, n, n_lobes,
                                       dict(optim.PAPER_LR, mean=float(np.float32(lr_mu))), t, **F32)
        torch.cuda.synchronize()
        got = planes.cpu().numpy()
        assert np.all(_close(got[:, :n], ref[:, :n], p_prev[:, :n])), t


@pytest.mark.parametrize("n", [1, 5000, 100_003])
def test_relocate_matches_oracle(n):
    """Sources bit-exact, copies bit-exact, new opacities to fp32 accuracy."""
    gc.ensure_built()
    rng = np.random.default_rng(n)
    n_lobes = 2
    NP = scenes.n_planes(n_lobes)
    pitch = scenes.round_pitch(n)
    p = rng.normal(size=(NP, pitch)).astype(np.float32)
    logit = rng.normal(0.0, 2.0, size=pitch).astype(np.float32)
    logit[rng.random(pitch) < 0.2] = -9.0                        # about a fifth are dead
    if n > 10:
        logit[3] = np.nan                                           # non-finite: dead
    p[10] = logit
    p[:, n:] = 5.0
    m = rng.normal(size=(NP, pitch)).astype(np.float32)
    rnd = rng.integers(0, 2 ** 32, size=n, dtype=np.uint64).astype(np.uint32)
    ref_p, ref_m, ref_v, ref_src, ref_k = optim.relocate(p, m, m, rnd.astype(np.uint64), n, 0.005)
    P = torch.from_numpy(p.copy()).cuda()
    opt = BetaAdam(P, n, n_lobes)
    opt.m.copy_(torch.from_numpy(m))
    opt.v.copy_(torch.from_numpy(m))
    count, src = opt.relocate(P, 0.005, torch.from_numpy(rnd.view(np.int32)).cuda())
    torch.cuda.synchronize()
    got_src = src.cpu().numpy()[:n]
    assert int(count.item()) == ref_k
    assert np.array_equal(got_src, ref_src)
    G = P.cpu().numpy()
    assert np.all(G[:, n:] == 5.0)
    keep = np.ones(NP, bool)
    keep[10] = False
    assert np.array_equal(G[keep, :n], ref_p[keep, :n].astype(np.float32))
    sig = lambda x: 1.0 / (1.0 + np.exp(-x.astype(np.float64)))
    assert np.allclose(sig(G[10, :n]), sig(ref_p[10, :n]), rtol=2e-6, atol=0)
    moved = ref_src >= 0
    assert np.all(opt.m.cpu().numpy()[:, :n][:, moved] == 0) and np.all(opt.v.cpu().numpy()[:, :n][:, moved] == 0)
    assert np.array_equal(opt.m.cpu().numpy()[:, :n][:, ~moved], m[:, :n][:, ~moved])
