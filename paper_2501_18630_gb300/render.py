"""PyTorch-side plumbing of the Beta rasterizer: device buffers, stream
handles and a torch.autograd.Function.  All arithmetic runs in
libbetasplat.so; this module only allocates memory and passes pointers.
"""
from __future__ import annotations

import ctypes
import math

import torch

from . import _lib
from .scenes import n_planes


def _vp(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else ctypes.c_void_p(0)


def _stream():
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


class Rasterizer:
    """Buffers and launches of project -> bin/sort -> raster fwd/bwd for one
    batch of views.  One forward may be in flight per instance: a second
    forward overwrites the saved per-pixel state of the first."""

    def __init__(self, n, pitch, n_lobes, cameras, opts: _lib.BetaOpts | None = None,
                 pair_capacity: int | None = None, device="cuda", persistent: bool = False,
                 hit_masks: bool = False):
        self.L = _lib.load()
        self.n, self.pitch, self.n_lobes = int(n), int(pitch), int(n_lobes)
        self.cameras = list(cameras)
        self.V = len(self.cameras)
        self.cams = _lib.make_cameras(self.cameras)
        self.opts = opts or _lib.default_opts()
        self.device = torch.device(device)
        L = self.L
        self.total_tiles = int(L.beta_total_tiles(self.cams, self.V, ctypes.byref(self.opts)))
        self.total_pixels = int(L.beta_total_pixels(self.cams, self.V))
        if self.total_tiles < 0 or self.total_pixels < 0:
            raise ValueError("invalid cameras or options")
        self.pix_off = []
        off = 0
        for c in self.cameras:
            self.pix_off.append(off)
            off += c.width * c.height
        dev = self.device
        self.proj = torch.empty(int(L.beta_proj_bytes(self.pitch, self.V)), dtype=torch.uint8, device=dev)
        self.ranges = torch.empty(self.total_tiles + 1, dtype=torch.int32, device=dev)
        self.count = torch.zeros(1, dtype=torch.int64, device=dev)
        self.status = torch.zeros(1, dtype=torch.int32, device=dev)
        self.color = torch.empty(3 * self.total_pixels, dtype=torch.float32, device=dev)
        self.T_final = torch.empty(self.total_pixels, dtype=torch.float32, device=dev)
        self.n_contrib = torch.empty(self.total_pixels, dtype=torch.int32, device=dev)
        # 2D-gradient accumulators: zero once here; beta_project_bwd re-clears them
        self.grad2d = torch.zeros(int(L.beta_grad2d_bytes(self.pitch, self.V)) // 4, dtype=torch.float32, device=dev)
        self.loss = torch.zeros(self.V, dtype=torch.float32, device=dev)
        self.dL_dcolor = torch.empty_like(self.color)
        self.l1_ws = torch.empty(max(4, int(L.beta_l1_workspace_bytes(self.cams, self.V))), dtype=torch.uint8, device=dev)
        nb = int(L.beta_raster_fwd_l1_workspace_bytes(self.cams, self.V, ctypes.byref(self.opts)))
        self.fwd_l1_ws = torch.empty(max(4, nb), dtype=torch.uint8, device=dev)
        # hit masks: the forward keeps which Betas may cover each pixel for the
        # backward (about 16 bytes per pixel on the sheet scenes); off, the
        # backward works them out again
        self.use_hit_masks = bool(hit_masks)
        self.hit_masks = None
        cap = pair_capacity if pair_capacity is not None else max(1 << 16, 4 * self.n * self.V)
        self._alloc_pairs(cap)
        self.persistent = bool(persistent)
        self.sched = None
        if self.persistent:
            nb = int(L.beta_schedule_bytes(self.cams, self.V, ctypes.byref(self.opts)))
            self.sched = torch.zeros(nb // 4, dtype=torch.int32, device=dev)

    # -- buffers -----------------------------------------------------------
    def _alloc_pairs(self, cap: int):
        cap = int(min(cap, 0x7FFFFFFF))
        self.cap = cap
        self.pair_vals = torch.empty(max(cap, 1), dtype=torch.int32, device=self.device)
        ws = int(self.L.beta_binsort_workspace_bytes(self.pitch, self.V, cap, self.cams, ctypes.byref(self.opts)))
        self.sort_ws = torch.empty(max(ws, 256), dtype=torch.uint8, device=self.device)
        if self.use_hit_masks:
            self.hit_masks = None
            nb = int(self.L.beta_hit_mask_bytes(self.cams, self.V, ctypes.byref(self.opts), cap))
            self.hit_masks = torch.empty(max(nb, 4) // 4, dtype=torch.int32, device=self.device)

    def _hm(self):
        if self.hit_masks is None:
            return ctypes.c_void_p(0), 0
        return _vp(self.hit_masks), self.hit_masks.numel() * 4

    def params(self, planes: torch.Tensor) -> _lib.BetaParams:
        assert planes.is_cuda and planes.dtype == torch.float32 and planes.is_contiguous()
        assert planes.shape == (n_planes(self.n_lobes), self.pitch), planes.shape
        return _lib.make_params(self.n, self.pitch, self.n_lobes, planes.data_ptr())

    def image(self, buf: torch.Tensor, v: int) -> torch.Tensor:
        """View v of a planar colour-like buffer as (3, H, W)."""
        c = self.cameras[v]
        o = 3 * self.pix_off[v]
        return buf[o:o + 3 * c.width * c.height].view(3, c.height, c.width)

    def plane(self, buf: torch.Tensor, v: int) -> torch.Tensor:
        c = self.cameras[v]
        o = self.pix_off[v]
        return buf[o:o + c.width * c.height].view(c.height, c.width)

    # -- the four steps ----------------------------------------------------
    def project(self, planes):
        prm = self.params(planes)
        _lib.check("beta_project", self.L.beta_project(ctypes.byref(prm), self.cams, self.V,
                                                        ctypes.byref(self.opts), _vp(self.proj), _stream()))

    def bin_sort(self, planes):
        prm = self.params(planes)
        _lib.check("beta_bin_sort", self.L.beta_bin_sort(
            ctypes.byref(prm), self.cams, self.V, ctypes.byref(self.opts), _vp(self.proj),
            _vp(self.pair_vals), self.cap, _vp(self.ranges), _vp(self.count), _vp(self.status),
            _vp(self.sort_ws), self.sort_ws.numel(), _stream()))

    def schedule(self):
        """Longest-first tile order for the persistent raster kernels."""
        _lib.check("beta_schedule", self.L.beta_schedule(
            self.cams, self.V, ctypes.byref(self.opts), _vp(self.ranges), _vp(self.sched),
            _vp(self.status), _stream()))

    def raster_fwd(self, planes):
        prm = self.params(planes)
        hm, hb = self._hm()
        _lib.check("beta_raster_fwd", self.L.beta_raster_fwd(
            ctypes.byref(prm), self.cams, self.V, ctypes.byref(self.opts), _vp(self.proj),
            _vp(self.pair_vals), _vp(self.ranges), _vp(self.sched), hm, hb, _vp(self.color),
            _vp(self.T_final), _vp(self.n_contrib), _vp(self.status), _stream()))

    def raster_fwd_l1(self, planes, target: torch.Tensor):
        """raster_fwd and l1_loss in one pass (the L1 term in the forward's epilogue)."""
        assert target.numel() == self.color.numel() and target.is_contiguous()
        prm = self.params(planes)
        hm, hb = self._hm()
        _lib.check("beta_raster_fwd_l1", self.L.beta_raster_fwd_l1(
            ctypes.byref(prm), self.cams, self.V, ctypes.byref(self.opts), _vp(self.proj),
            _vp(self.pair_vals), _vp(self.ranges), _vp(self.sched), hm, hb, _vp(self.color),
            _vp(self.T_final), _vp(self.n_contrib), _vp(target), _vp(self.loss), _vp(self.dL_dcolor),
            _vp(self.fwd_l1_ws), self.fwd_l1_ws.numel(), _vp(self.status), _stream()))
        return self.loss, self.dL_dcolor

    def l1_loss(self, target: torch.Tensor):
        assert target.numel() == self.color.numel() and target.is_contiguous()
        _lib.check("beta_l1_loss", self.L.beta_l1_loss(
            self.cams, self.V, _vp(self.color), _vp(target), _vp(self.loss), _vp(self.dL_dcolor),
            _vp(self.l1_ws), self.l1_ws.numel(), _stream()))
        return self.loss, self.dL_dcolor

    def dssim_loss(self, target: torch.Tensor, lambda_ssim: float = 0.2):
        """(1 - lambda) L1 + lambda (1 - SSIM) per view and its gradient (Sec. 3.4)."""
        assert target.numel() == self.color.numel() and target.is_contiguous()
        if getattr(self, "ssim_ws", None) is None:
            nb = int(self.L.beta_dssim_workspace_bytes(self.cams, self.V))
            self.ssim_ws = torch.empty(max(nb, 1), dtype=torch.uint8, device=self.color.device)
        _lib.check("beta_l1_dssim_loss", self.L.beta_l1_dssim_loss(
            self.cams, self.V, _vp(self.color), _vp(target), ctypes.c_float(lambda_ssim), _vp(self.loss),
            _vp(self.dL_dcolor), _vp(self.ssim_ws), self.ssim_ws.numel(), _stream()))
        return self.loss, self.dL_dcolor

    def raster_bwd(self, planes, dL_dcolor):
        prm = self.params(planes)
        assert dL_dcolor.numel() == self.color.numel() and dL_dcolor.is_contiguous()
        hm, hb = self._hm()
        _lib.check("beta_raster_bwd", self.L.beta_raster_bwd(
            ctypes.byref(prm), self.cams, self.V, ctypes.byref(self.opts), _vp(self.proj),
            _vp(self.pair_vals), _vp(self.ranges), _vp(self.sched), hm, hb, _vp(self.T_final),
            _vp(self.n_contrib), _vp(dL_dcolor), _vp(self.grad2d), _vp(self.status), _stream()))

    @property
    def fused_supported(self) -> bool:
        """Whether raster_fwd_bwd_l1 serves these options: every tile shape
        whose raster kernels give a thread two pixels, i.e. all but 8x4."""
        return bool(self.L.beta_raster_fwd_bwd_l1_supported(ctypes.byref(self.opts)))

    def raster_fwd_bwd_l1(self, planes, target: torch.Tensor, keep_state: bool = False):
        """raster_fwd_l1 followed by raster_bwd of its dL/dC, in one launch
        (each tile's CTA composites, forms the L1 term and walks back from its
        registers): colour, per-view loss and the 2D-gradient sums.  With
        keep_state T_final, n_contrib and dL_dcolor are written as well."""
        assert target.numel() == self.color.numel() and target.is_contiguous()
        prm = self.params(planes)
        keep = (lambda t: _vp(t)) if keep_state else (lambda t: ctypes.c_void_p(0))
        _lib.check("beta_raster_fwd_bwd_l1", self.L.beta_raster_fwd_bwd_l1(
            ctypes.byref(prm), self.cams, self.V, ctypes.byref(self.opts), _vp(self.proj),
            _vp(self.pair_vals), _vp(self.ranges), _vp(self.sched), _vp(self.color), keep(self.T_final),
            keep(self.n_contrib), _vp(target), _vp(self.loss), keep(self.dL_dcolor), _vp(self.grad2d),
            _vp(self.fwd_l1_ws), self.fwd_l1_ws.numel(), _vp(self.status), _stream()))
        return self.loss

    def project_bwd(self, planes, grad_planes, c0: int = 0, c1: int | None = None):
        """Raw-parameter gradients of primitives [c0, c1) (all by default): the
        same entry point on the primitive range, through pointers offset by c0
        (parameters, their gradients and the 2D-gradient slots, whose record
        index v * pitch + i keeps the full pitch)."""
        assert grad_planes.shape == planes.shape and grad_planes.is_contiguous()
        c1 = self.n if c1 is None else c1
        assert 0 <= c0 <= c1 <= self.n and c0 % 4 == 0
        assert planes.is_cuda and planes.dtype == torch.float32 and planes.is_contiguous()
        prm = _lib.make_params(c1 - c0, self.pitch, self.n_lobes, planes.data_ptr() + 4 * c0)
        _lib.check("beta_project_bwd", self.L.beta_project_bwd(
            ctypes.byref(prm), self.cams, self.V, ctypes.byref(self.opts),
            ctypes.c_void_p(self.grad2d.data_ptr() + 4 * 12 * c0),
            ctypes.c_void_p(grad_planes.data_ptr() + 4 * c0), _vp(self.status), _stream()))

    # -- composite calls ---------------------------------------------------
    def device_status(self):
        """(status, pair count); synchronises the current stream."""
        torch.cuda.current_stream().synchronize()
        return int(self.status.item()), int(self.count.item())

    def forward(self, planes, check_capacity: bool = True):
        """project + bin/sort + raster.  With check_capacity the pair count is
        read back (one host sync) and the pair buffers grow if needed."""
        self.project(planes)
        self.bin_sort(planes)
        if check_capacity:
            st, k = self.device_status()
            if st == _lib.BETA_ERR_CAPACITY:
                self._alloc_pairs(int(math.ceil(k * 1.25)) + 1024)
                self.bin_sort(planes)
                st, k = self.device_status()
            if st != _lib.BETA_OK:
                raise _lib.BetaError("beta_bin_sort", st, self.L.beta_status_string(st).decode())
        if self.persistent:
            self.schedule()
        self.raster_fwd(planes)
        return self.color

    def backward(self, planes, dL_dcolor, grad_planes=None):
        if grad_planes is None:
            grad_planes = torch.zeros_like(planes)
        self.raster_bwd(planes, dL_dcolor)
        self.project_bwd(planes, grad_planes)
        return grad_planes


class BetaRasterize(torch.autograd.Function):
    """colour = BetaRasterize.apply(planes, rasterizer): planar colour of every
    view (3 * total_pixels).  Backward returns d loss / d planes."""

    @staticmethod
    def forward(ctx, planes, rast: Rasterizer):
        color = rast.forward(planes).clone()
        ctx.rast = rast
        ctx.save_for_backward(planes)
        return color

    @staticmethod
    def backward(ctx, gcolor):
        (planes,) = ctx.saved_tensors
        grad = ctx.rast.backward(planes, gcolor.contiguous())
        return grad, None


def render(planes, rast: Rasterizer):
    return BetaRasterize.apply(planes, rast)
