"""Failure detection without a GPU fault: the scan's bounded look-back waits.

A scan block is told (through the host-side test hook beta_debug_scan_faults)
never to post its look-back entry, and the poll limit is made small, so the
blocks after it wait on an entry that nothing writes.  Each wait gives up
after the limit, the status word reads BETA_ERR_TIMEOUT, the kernels after
the scan skip their work (their outputs keep the caller's fill values), and
the next call with the default settings is exact again.
"""
import ctypes

import numpy as np
import pytest
import torch

import oracle
from paper_2501_18630_gb300 import _lib, render, scenes
from tests import gpu_common as gc

pytestmark = pytest.mark.gpu


@pytest.fixture
def L():
    gc.ensure_built()
    L = _lib.load()
    yield L
    assert L.beta_debug_scan_faults(0, -1) == _lib.BETA_OK   # defaults back, whatever happened


@pytest.mark.parametrize("withhold", [0, 3])
def test_scan_wait_runs_out_and_downstream_skips(L, withhold):
    sc = scenes.config_scene(3, n=30_000)
    cams = [scenes.ring_camera(4.0, 15.0, 0.3, 1920, 1080)]
    opts = _lib.default_opts(tile_w=16, tile_h=8, batch_s=128)
    planes = torch.from_numpy(sc.planes).cuda()
    rast = render.Rasterizer(sc.n, sc.pitch, sc.n_lobes, cams, opts)
    assert rast.total_tiles > 4 * 2048                  # several scan blocks, chained by look-back
    rast.forward(planes)                                # sizes the pair buffers
    st, K = rast.device_status()
    assert st == _lib.BETA_OK and K > 0

    assert L.beta_debug_scan_faults(2000, withhold) == _lib.BETA_OK
    rast.pair_vals.fill_(-7)
    rast.color.fill_(-3.0)
    rast.project(planes)
    rast.bin_sort(planes)
    rast.raster_fwd(planes)
    torch.cuda.synchronize()
    st, _ = rast.device_status()
    assert st == _lib.BETA_ERR_TIMEOUT
    assert bool((rast.pair_vals == -7).all())           # scatter and list sort wrote nothing
    assert bool((rast.color == -3.0).all())             # the raster forward skipped its work

    assert L.beta_debug_scan_faults(0, -1) == _lib.BETA_OK
    rast.forward(planes)
    st, K2 = rast.device_status()
    assert st == _lib.BETA_OK and K2 == K
    K3, ranges, vals = gc.sorted_pairs(rast)
    _, recs, oranges = oracle.bin_pairs(sc.planes, sc.n, sc.n_lobes, cams, tile_w=16, tile_h=8, pitch=sc.pitch)
    assert np.array_equal(ranges, oranges) and np.array_equal(vals, recs)
