"""The optimiser step that follows the rasterizer's backward (Sec. 3.4):
Adam on the raw parameters with the composite loss's opacity and scale
regularisers and the Beta-kernel-scaled position noise, one launch of
beta_adam_step per step.  State (moments, step count) lives on the device."""
from __future__ import annotations

import ctypes

import torch

from . import _lib


class BetaAdam:
    """Adam state for SoA parameter planes [(15 + 6M), pitch] (float32, CUDA).

    step(planes, grad) updates planes in place; eta (3 x pitch standard
    normal samples for the position noise) is drawn with torch.randn unless
    given; lr_mean overrides the position learning rate (the caller's decay
    schedule).  reg_loss holds the running sum of the two regulariser values
    (lambda_o sum o, lambda_Sigma sum s) added by each step."""

    def __init__(self, planes: torch.Tensor, n: int, n_lobes: int, lr: dict | None = None, **opts):
        self.n, self.n_lobes, self.pitch = n, n_lobes, planes.shape[1]
        self.m = torch.zeros_like(planes)
        self.v = torch.zeros_like(planes)
        self.reg_loss = torch.zeros(2, dtype=torch.float64, device=planes.device)
        self.opts = _lib.adam_default_opts(lr, **opts)
        self.t = 0

    def step(self, planes: torch.Tensor, grad: torch.Tensor, eta: torch.Tensor | None = None,
             lr_mean: float | None = None):
        if eta is None:
            eta = torch.randn(3, self.pitch, dtype=torch.float32, device=planes.device)
        self.t += 1
        self.opts.step = self.t
        if lr_mean is not None:
            self.opts.lr[0] = lr_mean
        vp = lambda t: ctypes.c_void_p(t.data_ptr())
        _lib.check("beta_adam_step", _lib.load().beta_adam_step(
            self.n, self.pitch, self.n_lobes, vp(planes), vp(grad), vp(self.m), vp(self.v), vp(eta),
            ctypes.byref(self.opts), vp(self.reg_loss),
            ctypes.c_void_p(torch.cuda.current_stream(planes.device).cuda_stream)))
        return planes

    def relocate(self, planes: torch.Tensor, min_opacity: float = 0.005, rnd: torch.Tensor | None = None):
        """Respawns dead primitives as copies of live ones (Sec. 3.4
        Densification); returns (number relocated, source index per
        primitive) as device tensors.  rnd: [n] uniform 32-bit words
        (int32 tensor, reinterpreted), drawn with torch.randint if absent."""
        dev = planes.device
        if rnd is None:
            rnd = torch.randint(-2 ** 31, 2 ** 31, (max(self.n, 1),), dtype=torch.int32, device=dev)
        L = _lib.load()
        ws = torch.empty(max(1, int(L.beta_relocate_workspace_bytes(self.n))), dtype=torch.uint8, device=dev)
        src = torch.empty(max(self.n, 1), dtype=torch.int32, device=dev)
        count = torch.zeros(1, dtype=torch.int32, device=dev)
        vp = lambda t: ctypes.c_void_p(t.data_ptr())
        _lib.check("beta_relocate", L.beta_relocate(
            self.n, self.pitch, self.n_lobes, vp(planes), vp(self.m), vp(self.v), vp(rnd),
            ctypes.c_float(min_opacity), vp(ws), ws.numel(), vp(src), vp(count),
            ctypes.c_void_p(torch.cuda.current_stream(dev).cuda_stream)))
        return count, src
