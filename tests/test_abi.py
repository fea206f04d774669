"""The C-ABI library builds, loads and exports every symbol include/*.h
declares; host-only queries and argument checks work without a GPU."""
import ctypes
import glob
import math
import os
import re

import pytest

from paper_2501_18630_gb300 import _lib, build, scenes

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    build.build()
    return _lib.load()


def declared_symbols():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        for m in re.finditer(r"\b(beta_[a-z0-9_]+)\s*\(", src):
            names.add(m.group(1))
    return sorted(names)


def test_every_declared_symbol_is_exported(L):
    names = declared_symbols()
    assert len(names) >= 14
    for name in names:
        assert hasattr(L, name), name
    assert set(_lib.EXPORTS) <= set(names)


def test_header_prototypes_match_binding(L):
    # the binding declares every exported entry point
    for name in declared_symbols():
        assert getattr(L, name).argtypes is not None or name in ("beta_version",), name


def test_adam_defaults_are_the_papers(L):
    ao = _lib.adam_default_opts()
    lr = dict(zip(_lib.ADAM_GROUPS, list(ao.lr)))
    assert lr["mean"] == pytest.approx(1.6e-4) and lr["opacity"] == pytest.approx(0.05)
    assert lr["log_scale"] == pytest.approx(5e-3) and lr["quat"] == pytest.approx(1e-3)
    assert lr["b"] == pytest.approx(1e-3) and lr["c0"] == pytest.approx(2.5e-3)
    assert ao.lambda_o == pytest.approx(0.01) and ao.lambda_sigma == pytest.approx(0.01)
    assert ao.lambda_eps == pytest.approx(5e4) and ao.noise_b == pytest.approx(math.log(25.0))


def test_host_queries(L):
    o = _lib.default_opts()
    assert (o.tile_w, o.tile_h, o.batch_s, o.color_mode) == (16, 16, 256, 0)
    assert o.t_eps == pytest.approx(2.0 ** -19) and o.alpha_max == pytest.approx(0.99)
    assert math.isinf(o.b_lo) and o.b_lo < 0 and math.isinf(o.b_hi)
    assert L.beta_version() >= 1
    cams = [scenes.pinhole(*scenes.look_at((0, 0, -3)), 1297, 840),
            scenes.pinhole(*scenes.look_at((0, 0, -3)), 256, 256)]
    arr = _lib.make_cameras(cams)
    assert L.beta_total_tiles(arr, 2, ctypes.byref(o)) == 82 * 53 + 16 * 16
    assert L.beta_total_pixels(arr, 2) == 1297 * 840 + 256 * 256
    assert L.beta_proj_bytes(1024, 3) == 1024 * 3 * 68 + 16
    assert L.beta_proj_bytes(1000, 2) == 1000 * 2 * 64 + 1024 * 2 * 4 + 16
    assert L.beta_grad2d_bytes(1024, 2) == 1024 * 2 * 48
    assert L.beta_binsort_workspace_bytes(1024, 2, 10000, arr, ctypes.byref(o)) > 0
    assert L.beta_l1_workspace_bytes(arr, 2) >= 4 * ((1297 * 840 + 255) // 256)
    for code in (0, -1, -2, -3, -4, -5, -6):
        assert L.beta_status_string(code)
    # hit masks: per 32 pairs of capacity and per tile, one word per lane (a pixel pair in
    # tiles of whole 16x4 / 8x8 pair blocks, a pixel in 8x4 tiles) and one per warp
    tiles = 82 * 53 + 16 * 16
    assert L.beta_hit_mask_bytes(arr, 2, ctypes.byref(o), 10000) == ((10000 >> 5) + tiles + 1) * (128 + 4) * 4
    o84 = _lib.default_opts(tile_w=8, tile_h=4)
    tiles84 = 163 * 210 + 32 * 64
    assert L.beta_total_tiles(arr, 2, ctypes.byref(o84)) == tiles84
    assert L.beta_hit_mask_bytes(arr, 2, ctypes.byref(o84), 10000) == ((10000 >> 5) + tiles84 + 1) * (32 + 1) * 4
    o88 = _lib.default_opts(tile_w=8, tile_h=8)
    tiles88 = 163 * 105 + 32 * 32
    assert L.beta_hit_mask_bytes(arr, 2, ctypes.byref(o88), 10000) == ((10000 >> 5) + tiles88 + 1) * (32 + 1) * 4
    assert L.beta_hit_mask_bytes(arr, 2, ctypes.byref(o), -1) == 0


def test_argument_errors_are_returned_without_launch(L):
    o = _lib.default_opts()
    cams = _lib.make_cameras([scenes.pinhole(*scenes.look_at((0, 0, -3)), 64, 64)])
    prm = _lib.make_params(10, 32, 1, 0x1000)
    # null projection buffer
    assert L.beta_project(ctypes.byref(prm), cams, 1, ctypes.byref(o), None, None) == _lib.BETA_ERR_ARG
    # pitch not a multiple of 4
    bad = _lib.make_params(10, 30, 1, 0x1000)
    assert L.beta_project(ctypes.byref(bad), cams, 1, ctypes.byref(o), ctypes.c_void_p(0x2000), None) == _lib.BETA_ERR_ARG
    # too many lobes
    bad = _lib.make_params(10, 32, 9, 0x1000)
    assert L.beta_project(ctypes.byref(bad), cams, 1, ctypes.byref(o), ctypes.c_void_p(0x2000), None) == _lib.BETA_ERR_ARG
    # unsupported tile shape
    o2 = _lib.default_opts(tile_w=8)
    assert L.beta_project(ctypes.byref(prm), cams, 1, ctypes.byref(o2), ctypes.c_void_p(0x2000), None) == _lib.BETA_ERR_UNSUPPORTED
    # zero views
    assert L.beta_project(ctypes.byref(prm), cams, 0, ctypes.byref(o), ctypes.c_void_p(0x2000), None) == _lib.BETA_ERR_ARG
    # workspace too small
    vp = ctypes.c_void_p(0x2000)
    r = L.beta_bin_sort(ctypes.byref(prm), cams, 1, ctypes.byref(o), vp, vp, 100, vp, vp, vp, vp, 16, None)
    assert r == _lib.BETA_ERR_WORKSPACE
    # capacity beyond 2^31 - 1
    r = L.beta_bin_sort(ctypes.byref(prm), cams, 1, ctypes.byref(o), vp, vp, 1 << 31, vp, vp, vp, vp, 1 << 40, None)
    assert r == _lib.BETA_ERR_ARG
    # optimiser step: null pointers, n > pitch, step < 1
    ao = _lib.adam_default_opts()
    assert L.beta_adam_step(10, 32, 1, None, vp, vp, vp, vp, ctypes.byref(ao), None, None) == _lib.BETA_ERR_ARG
    assert L.beta_adam_step(40, 32, 1, vp, vp, vp, vp, vp, ctypes.byref(ao), None, None) == _lib.BETA_ERR_ARG
    ao.step = 0
    assert L.beta_adam_step(10, 32, 1, vp, vp, vp, vp, vp, ctypes.byref(ao), None, None) == _lib.BETA_ERR_ARG
    # invalid alpha_max
    o3 = _lib.default_opts(alpha_max=1.0)
    assert L.beta_project(ctypes.byref(prm), cams, 1, ctypes.byref(o3), vp, None) == _lib.BETA_ERR_ARG


def test_product_path_has_no_cpu_fallback():
    """The package never imports the oracle, and the binding raises when the
    library file is absent."""
    pkg = os.path.join(ROOT, "paper_2501_18630_gb300")
    for f in glob.glob(os.path.join(pkg, "*.py")):
        src = open(f).read()
        assert "import oracle" not in src and "from oracle" not in src, f
    with pytest.raises(RuntimeError):
        saved = _lib._lib
        try:
            _lib._lib = None
            _lib.load(os.path.join(ROOT, "does-not-exist.so"))
        finally:
            _lib._lib = saved


def test_scan_fault_hook_checks_its_arguments(L):
    """The look-back fault-injection hook is host-only: it validates its
    arguments and stores them for later launches (no device work)."""
    assert L.beta_debug_scan_faults(-1, -1) == _lib.BETA_ERR_ARG
    assert L.beta_debug_scan_faults((1 << 20) + 1, -1) == _lib.BETA_ERR_ARG
    assert L.beta_debug_scan_faults(100, -2) == _lib.BETA_ERR_ARG
    assert L.beta_debug_scan_faults(100, 3) == _lib.BETA_OK
    assert L.beta_debug_scan_faults(0, -1) == _lib.BETA_OK      # defaults restored


def test_static_scratch_size_matches_header():
    """The binding's copy of the static-scratch size is read from the header."""
    src = open(os.path.join(ROOT, "include", "beta_splat.h")).read()
    m = re.search(r"#define\s+BETA_STATIC_SCRATCH_BYTES\s+\((\d+)u \* (\d+)u \* (\d+)u\)", src)
    assert m and _lib.STATIC_SCRATCH_BYTES == int(m.group(1)) * int(m.group(2)) * int(m.group(3))


def test_one_launch_raster_support_and_argument_errors(L):
    """beta_raster_fwd_bwd_l1 serves every tile shape with pixel-pair kernels
    (not 8x4), and refuses bad arguments before anything is launched."""
    for (tw, th), want in (((16, 16), 1), ((16, 8), 1), ((8, 8), 1), ((32, 16), 1), ((8, 4), 0), ((8, 16), 0)):
        o = _lib.default_opts(tile_w=tw, tile_h=th)
        assert L.beta_raster_fwd_bwd_l1_supported(ctypes.byref(o)) == want, (tw, th)
    assert L.beta_raster_fwd_bwd_l1_supported(ctypes.byref(_lib.default_opts(alpha_max=1.0))) == 0
    cams = _lib.make_cameras([scenes.pinhole(*scenes.look_at((0, 0, -3)), 64, 64)])
    prm = _lib.make_params(10, 32, 1, 0x1000)
    vp = ctypes.c_void_p(0x2000)
    o = _lib.default_opts(tile_w=16, tile_h=8)

    def call(opts, target=vp, grad2d=vp, ws=vp, ws_bytes=1 << 20):
        return L.beta_raster_fwd_bwd_l1(ctypes.byref(prm), cams, 1, ctypes.byref(opts), vp, vp, vp, None, vp,
                                        None, None, target, vp, None, grad2d, ws, ws_bytes, vp, None)

    assert call(o, target=None) == _lib.BETA_ERR_ARG                         # no target
    assert call(o, grad2d=ctypes.c_void_p(0x2004)) == _lib.BETA_ERR_ARG      # grad2d not 16-byte aligned
    assert call(_lib.default_opts(tile_w=8, tile_h=4)) == _lib.BETA_ERR_ARG  # no pixel-pair kernels
    assert call(o, ws=None) == _lib.BETA_ERR_WORKSPACE
    assert call(o, ws_bytes=4) == _lib.BETA_ERR_WORKSPACE                    # one float per tile needed
