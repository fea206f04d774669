"""The L1 + DSSIM loss (beta_l1_dssim_loss) against the FP64 oracle
(oracle.ssim), through the C ABI: per-view losses and dL/dC element by
element on ragged multi-view batches, lambda 0 (plain L1) and 1 (SSIM only),
identical images, and the gradient through the rasterizer's backward."""
import ctypes

import numpy as np
import pytest
import torch

from oracle import ssim
from paper_2501_18630_gb300 import _lib, scenes
from tests import gpu_common as gc

pytestmark = pytest.mark.gpu


def _run(cams, color, target, lam):
    gc.ensure_built()
    L = _lib.load()
    arr = _lib.make_cameras(cams)
    V = len(cams)
    nb = int(L.beta_dssim_workspace_bytes(arr, V))
    ws = torch.empty(nb, dtype=torch.uint8, device="cuda")
    c = torch.from_numpy(color.astype(np.float32)).cuda()
    t = torch.from_numpy(target.astype(np.float32)).cuda()
    loss = torch.zeros(V, dtype=torch.float32, device="cuda")
    d = torch.zeros_like(c)
    vp = lambda x: ctypes.c_void_p(x.data_ptr())
    _lib.check("beta_l1_dssim_loss", L.beta_l1_dssim_loss(arr, V, vp(c), vp(t), ctypes.c_float(lam), vp(loss),
                                                          vp(d), vp(ws), nb, None))
    torch.cuda.synchronize()
    return loss.cpu().numpy(), d.cpu().numpy()


def _views(cams, flat):
    out, off = [], 0
    for cam in cams:
        n = 3 * cam.width * cam.height
        out.append(flat[off:off + n].reshape(3, cam.height, cam.width))
        off += n
    return out


@pytest.mark.parametrize("lam", [0.2, 0.0, 1.0])
def test_loss_and_gradient_match_oracle(lam):
    rng = np.random.default_rng(3)
    cams = [scenes.pinhole(*scenes.look_at((0, 0, -3)), w, h) for (w, h) in ((70, 45), (33, 17), (128, 64))]
    npx = sum(3 * c.width * c.height for c in cams)
    target = rng.random(npx)
    color = np.clip(target + rng.normal(0.0, 0.1, npx), 0.0, 1.0)
    color[:50] = target[:50]                                  # ties: sign(0) = 0
    loss, d = _run(cams, color, target, lam)
    for v, (cx, ty, dv) in enumerate(zip(_views(cams, color), _views(cams, target), _views(cams, d))):
        assert loss[v] == pytest.approx(ssim.loss(cx, ty, lam), rel=2e-5, abs=1e-7)
        ref = ssim.grad(cx, ty, lam)
        scale = np.abs(ref).max()
        assert np.abs(dv - ref).max() <= 2e-4 * scale, (v, np.abs(dv - ref).max(), scale)


def test_identical_images_have_zero_ssim_loss():
    rng = np.random.default_rng(4)
    cams = [scenes.pinhole(*scenes.look_at((0, 0, -3)), 96, 50)]
    img = rng.random(3 * 96 * 50)
    loss, d = _run(cams, img, img, 0.2)
    assert abs(loss[0]) < 1e-6 and np.abs(d).max() < 1e-8


def test_full_hd_view_sampled():
    """One 1920x1080 view at the bench resolution: loss to the oracle, and the
    gradient on sampled pixels (the oracle's filter over the whole view)."""
    rng = np.random.default_rng(5)
    cams = [scenes.pinhole(*scenes.look_at((0, 0, -3)), 1920, 1080)]
    target = rng.random(3 * 1920 * 1080)
    color = np.clip(target + rng.normal(0.0, 0.05, target.size), 0.0, 1.0)
    loss, d = _run(cams, color, target, 0.2)
    cx, ty = color.reshape(3, 1080, 1920), target.reshape(3, 1080, 1920)
    assert loss[0] == pytest.approx(ssim.loss(cx, ty, 0.2), rel=2e-5)
    ref = ssim.grad(cx, ty, 0.2)
    idx = rng.integers(0, ref.size, 20000)
    dv = d.reshape(-1)[idx]
    rv = ref.reshape(-1)[idx]
    assert np.abs(dv - rv).max() <= 2e-4 * np.abs(ref).max()
