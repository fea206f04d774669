"""Batched forward + backward of many views as one replayable CUDA graph.

The whole step -- project, bin/sort, longest-first schedule, raster forward
with the per-view L1 loss in its epilogue, raster backward (for the tile
shapes with pixel-pair kernels both in one launch, beta_raster_fwd_bwd_l1),
projection backward -- is captured once and replayed.  Every entry point only enqueues
kernels and the pair count stays on the device, so nothing in the step
synchronises with the host.  A pair-capacity overflow shows up in the device
status word; check() reads it (one sync), grows the buffers and recaptures.
"""
from __future__ import annotations

import math

import torch

from . import _lib
from .render import Rasterizer


class BatchedStep:
    def __init__(self, planes: torch.Tensor, n: int, n_lobes: int, cameras, target: torch.Tensor,
                 opts: _lib.BetaOpts | None = None, persistent: bool = True, headroom: float = 1.15,
                 hit_masks: bool = True, graph_project_bwd: bool = True, fused: bool = True):
        """graph_project_bwd=False leaves the projection backward out of the
        captured graph, for project_bwd_reduced() to run it in chunks, each
        chunk's gradient all-reduce overlapping the next chunk.  fused=False
        runs the raster forward (+ L1) and backward as two launches even where
        the one-launch kernel exists; hit masks only serve that split path."""
        self.planes = planes
        self.target = target
        self.graph_project_bwd = bool(graph_project_bwd)
        self.rast = Rasterizer(n, planes.shape[1], n_lobes, cameras, opts, device=planes.device,
                               persistent=persistent)
        self.fused = bool(fused) and self.rast.fused_supported
        self.rast.use_hit_masks = bool(hit_masks) and not self.fused   # allocated by _size_pairs
        self.grad = torch.zeros_like(planes)
        self.headroom = headroom
        self.graph = None
        self._size_pairs()

    def _size_pairs(self):
        r = self.rast
        r.forward(self.planes, check_capacity=True)
        _, k = r.device_status()
        r._alloc_pairs(int(math.ceil(k * self.headroom)) + 65536)

    def body(self):
        """The step as eager launches on the current stream."""
        r = self.rast
        r.project(self.planes)
        r.bin_sort(self.planes)
        if r.persistent:
            r.schedule()
        if self.fused:
            r.raster_fwd_bwd_l1(self.planes, self.target)
        else:
            r.raster_fwd_l1(self.planes, self.target)
            r.raster_bwd(self.planes, r.dL_dcolor)
        if self.graph_project_bwd:
            r.project_bwd(self.planes, self.grad)

    def project_bwd_reduced(self, chunk: int | None = None):
        """Projection backward in chunks of primitives, each chunk's gradient
        summed over the ranks by an asynchronous all-reduce that overlaps the
        next chunks (after a step() captured with graph_project_bwd=False)."""
        from .distributed import reduce_gradients_chunked
        r = self.rast
        chunk = chunk or max(4, (r.n + 7) // 8)
        return reduce_gradients_chunked(self.grad, lambda c0, c1: r.project_bwd(self.planes, self.grad, c0, c1),
                                        r.n, chunk)

    def capture(self):
        side = torch.cuda.Stream(device=self.planes.device)
        side.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(side):
            self.body()                       # warm-up outside the graph (lazy module loading)
            if not self.graph_project_bwd:
                # consume the warm-up's 2D-gradient sums (the projection backward clears them)
                self.rast.project_bwd(self.planes, self.grad)
        torch.cuda.current_stream().wait_stream(side)
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            self.body()
        self.graph = g
        return g

    def step(self):
        if self.graph is None:
            self.capture()
        self.graph.replay()

    def check(self) -> int:
        """Reads the device status after a replay; on a capacity overflow grows
        the pair buffers, recaptures and replays.  Returns the pair count."""
        st, k = self.rast.device_status()
        if st == _lib.BETA_ERR_CAPACITY:
            self.rast._alloc_pairs(int(math.ceil(k * self.headroom)) + 65536)
            self.graph = None
            self.step()
            if not self.graph_project_bwd:
                self.project_bwd_reduced()
            st, k = self.rast.device_status()
        if st != _lib.BETA_OK:
            raise _lib.BetaError("batched step", st, _lib.load().beta_status_string(st).decode())
        return k

    @property
    def loss(self):
        return self.rast.loss
