"""beta_bin_sort_static: the binning + sort step for callers that cannot
allocate device memory (a plugin whose host application owns every device
allocation, a real-time loop that must not hit cudaMalloc's implicit
synchronisation, a deployment that reserves all memory at load time).  It
takes its workspace from a fixed array inside the library instead of from
the caller.

The test calls it through the C ABI twice in a row, on two different
problems, and checks its outputs against beta_bin_sort with a caller
workspace.  Binning is integer work, so the comparison is bit-exact (the
tolerance every binning test here uses).  Kept in a file that pytest
collects last, and self-contained so it also passes alone.
"""
import ctypes

import numpy as np
import pytest
import torch

from paper_2501_18630_gb300 import _lib, build, render, scenes

pytestmark = pytest.mark.gpu


def _vp(t):
    return ctypes.c_void_p(t.data_ptr())


def _static_bin_sort(rast, planes):
    L = _lib.load()
    prm = rast.params(planes)
    vals = torch.full((rast.cap,), -7, dtype=torch.int32, device="cuda")
    ranges = torch.full((rast.total_tiles + 1,), -7, dtype=torch.int32, device="cuda")
    count = torch.full((1,), -7, dtype=torch.int64, device="cuda")
    status = torch.full((1,), -7, dtype=torch.int32, device="cuda")
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    code = L.beta_bin_sort_static(ctypes.byref(prm), rast.cams, rast.V, ctypes.byref(rast.opts),
                                  _vp(rast.proj), _vp(vals), rast.cap, _vp(ranges), _vp(count),
                                  _vp(status), stream)
    torch.cuda.synchronize()
    return code, vals, ranges, count, status


def test_static_scratch_bin_sort_matches_workspace_version():
    build.build()
    L = _lib.load()
    problems = [
        # larger problem first, then a smaller one: stale scratch contents of
        # the first call must not leak into the second
        (scenes.config_scene(2, n=120_000), [scenes.ring_camera(4.0, 20.0, 0.3, 800, 600),
                                             scenes.ring_camera(4.0, 20.0, 1.9, 640, 480)]),
        (scenes.config_scene(1, n=4096), None),
    ]
    for sc, cams in problems:
        cams = cams or sc.cameras
        planes = torch.from_numpy(sc.planes).cuda()
        rast = render.Rasterizer(sc.n, sc.pitch, sc.n_lobes, cams)
        rast.forward(planes, check_capacity=True)           # sizes the pair buffers
        st, K = rast.device_status()
        assert st == 0 and K > 0
        need = L.beta_binsort_workspace_bytes(rast.pitch, rast.V, rast.cap, rast.cams, ctypes.byref(rast.opts))
        assert 0 < need <= _lib.STATIC_SCRATCH_BYTES
        ref_vals = rast.pair_vals[:K].cpu().numpy().copy()
        ref_ranges = rast.ranges.cpu().numpy().copy()
        code, vals, ranges, count, status = _static_bin_sort(rast, planes)
        assert code == _lib.BETA_OK
        assert int(status.item()) == 0 and int(count.item()) == K
        assert np.array_equal(ranges.cpu().numpy(), ref_ranges)
        assert np.array_equal(vals[:K].cpu().numpy(), ref_vals)


def test_static_scratch_rejects_problems_beyond_its_size():
    build.build()
    L = _lib.load()
    sc = scenes.config_scene(1, n=4096)
    cam = sc.cameras[0]
    planes = torch.from_numpy(sc.planes).cuda()
    rast = render.Rasterizer(sc.n, sc.pitch, sc.n_lobes, [cam], pair_capacity=4_000_000)
    need = L.beta_binsort_workspace_bytes(rast.pitch, 1, rast.cap, rast.cams, ctypes.byref(rast.opts))
    assert need > _lib.STATIC_SCRATCH_BYTES
    rast.project(planes)
    code, vals, ranges, count, status = _static_bin_sort(rast, planes)
    assert code == _lib.BETA_ERR_WORKSPACE
    # nothing was launched: the outputs keep their fill values
    assert int(status.item()) == -7 and int(count.item()) == -7
