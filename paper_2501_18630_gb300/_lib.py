"""ctypes binding of libbetasplat.so (include/beta_splat.h).

Argument marshalling only: every computation runs in the CUDA library.  If
the library is missing the import of any entry point raises, so no CPU
fallback can ever stand in for it.
"""
from __future__ import annotations

import ctypes
import math
import os
import threading

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libbetasplat.so")

BETA_OK = 0
BETA_ERR_ARG = -1
BETA_ERR_CAPACITY = -2
BETA_ERR_CUDA = -3
BETA_ERR_TIMEOUT = -4
BETA_ERR_UNSUPPORTED = -5
BETA_ERR_WORKSPACE = -6
MAX_LOBES = 8
MAX_VIEWS = 64


def _header_define(name: str) -> int:
    """Integer value of a #define in include/beta_splat.h (unsigned suffixes dropped)."""
    import re
    hdr = os.path.join(os.path.dirname(HERE), "include", "beta_splat.h")
    m = re.search(r"^#define\s+" + name + r"\s+(.+)$", open(hdr).read(), re.M)
    if not m:
        raise RuntimeError(f"{name} is not defined in {hdr}")
    expr = re.sub(r"(\d+)[uUlL]+", r"\1", m.group(1).split("/*")[0].strip())
    if not re.fullmatch(r"[\d\s*()+<]+", expr):
        raise RuntimeError(f"{name}: unexpected expression {expr!r}")
    return int(eval(expr, {"__builtins__": {}}))


# size of the library's own scratch array behind beta_bin_sort_static
STATIC_SCRATCH_BYTES = _header_define("BETA_STATIC_SCRATCH_BYTES")

EXPORTS = [
    "beta_default_opts", "beta_status_string", "beta_version", "beta_proj_bytes",
    "beta_total_tiles", "beta_total_pixels", "beta_binsort_workspace_bytes", "beta_grad2d_bytes",
    "beta_l1_workspace_bytes", "beta_project", "beta_bin_sort", "beta_raster_fwd", "beta_l1_loss",
    "beta_raster_bwd", "beta_project_bwd", "beta_bin_sort_static", "beta_schedule_bytes",
    "beta_schedule", "beta_adam_default_opts", "beta_adam_step", "beta_relocate_workspace_bytes",
    "beta_relocate", "beta_dssim_workspace_bytes", "beta_l1_dssim_loss",
    "beta_raster_fwd_l1_workspace_bytes", "beta_raster_fwd_l1", "beta_debug_scan_faults",
    "beta_hit_mask_bytes", "beta_raster_fwd_bwd_l1", "beta_raster_fwd_bwd_l1_supported",
]


class BetaParams(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int32), ("pitch", ctypes.c_int32), ("n_lobes", ctypes.c_int32),
                ("reserved", ctypes.c_int32), ("planes", ctypes.c_void_p)]


class BetaCamera(ctypes.Structure):
    _fields_ = [("R", ctypes.c_float * 9), ("t", ctypes.c_float * 3), ("fx", ctypes.c_float),
                ("fy", ctypes.c_float), ("cx", ctypes.c_float), ("cy", ctypes.c_float),
                ("near_plane", ctypes.c_float), ("width", ctypes.c_int32), ("height", ctypes.c_int32),
                ("bg", ctypes.c_float * 3)]


class BetaOpts(ctypes.Structure):
    _fields_ = [("tile_w", ctypes.c_int32), ("tile_h", ctypes.c_int32), ("batch_s", ctypes.c_int32),
                ("color_mode", ctypes.c_int32), ("t_eps", ctypes.c_float), ("alpha_max", ctypes.c_float),
                ("blur_eps", ctypes.c_float), ("b_lo", ctypes.c_float), ("b_hi", ctypes.c_float)]


class BetaAdamOpts(ctypes.Structure):
    _fields_ = [("lr", ctypes.c_float * 9), ("beta1", ctypes.c_float), ("beta2", ctypes.c_float),
                ("eps", ctypes.c_float), ("lambda_o", ctypes.c_float), ("lambda_sigma", ctypes.c_float),
                ("lambda_eps", ctypes.c_float), ("noise_b", ctypes.c_float), ("step", ctypes.c_int32)]


# learning-rate groups of BetaAdamOpts.lr, in order
ADAM_GROUPS = ("mean", "log_scale", "quat", "opacity", "b", "c0", "lobe_dir", "lobe_b", "lobe_color")


class BetaError(RuntimeError):
    def __init__(self, fn, code, msg):
        super().__init__(f"{fn} failed: {code} ({msg})")
        self.code = code


_lock = threading.Lock()
_lib = None


def load(path: str = LIB_PATH):
    """Load libbetasplat.so and declare the prototypes.  Raises if missing."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(path):
            raise RuntimeError(
                f"{path} is not built: run `python -c 'import __graft_entry__ as g; g.build()'`")
        L = ctypes.CDLL(path)
        vp, sz, i32, i64 = ctypes.c_void_p, ctypes.c_size_t, ctypes.c_int32, ctypes.c_int64
        P, C, O = ctypes.POINTER(BetaParams), ctypes.POINTER(BetaCamera), ctypes.POINTER(BetaOpts)
        sig = {
            "beta_default_opts": (None, [O]),
            "beta_status_string": (ctypes.c_char_p, [ctypes.c_int]),
            "beta_version": (i32, []),
            "beta_debug_scan_faults": (ctypes.c_int, [i32, i64]),
            "beta_proj_bytes": (sz, [i32, i32]),
            "beta_total_tiles": (i64, [C, i32, O]),
            "beta_total_pixels": (i64, [C, i32]),
            "beta_binsort_workspace_bytes": (sz, [i32, i32, i64, C, O]),
            "beta_grad2d_bytes": (sz, [i32, i32]),
            "beta_l1_workspace_bytes": (sz, [C, i32]),
            "beta_project": (ctypes.c_int, [P, C, i32, O, vp, vp]),
            "beta_bin_sort": (ctypes.c_int, [P, C, i32, O, vp, vp, i64, vp, vp, vp, vp, sz, vp]),
            "beta_hit_mask_bytes": (sz, [C, i32, O, i64]),
            "beta_raster_fwd": (ctypes.c_int, [P, C, i32, O, vp, vp, vp, vp, vp, sz, vp, vp, vp, vp, vp]),
            "beta_l1_loss": (ctypes.c_int, [C, i32, vp, vp, vp, vp, vp, sz, vp]),
            "beta_raster_fwd_l1_workspace_bytes": (sz, [C, i32, O]),
            "beta_raster_fwd_l1": (ctypes.c_int, [P, C, i32, O, vp, vp, vp, vp, vp, sz, vp, vp, vp, vp, vp,
                                                  vp, vp, sz, vp, vp]),
            "beta_raster_bwd": (ctypes.c_int, [P, C, i32, O, vp, vp, vp, vp, vp, sz, vp, vp, vp, vp, vp, vp]),
            "beta_raster_fwd_bwd_l1": (ctypes.c_int, [P, C, i32, O, vp, vp, vp, vp, vp, vp, vp, vp, vp, vp,
                                                      vp, vp, sz, vp, vp]),
            "beta_raster_fwd_bwd_l1_supported": (ctypes.c_int, [O]),
            "beta_schedule_bytes": (sz, [C, i32, O]),
            "beta_schedule": (ctypes.c_int, [C, i32, O, vp, vp, vp, vp]),
            "beta_project_bwd": (ctypes.c_int, [P, C, i32, O, vp, vp, vp, vp]),
            "beta_bin_sort_static": (ctypes.c_int, [P, C, i32, O, vp, vp, i64, vp, vp, vp, vp]),
            "beta_adam_default_opts": (None, [ctypes.POINTER(BetaAdamOpts)]),
            "beta_adam_step": (ctypes.c_int, [i32, i32, i32, vp, vp, vp, vp, vp,
                                              ctypes.POINTER(BetaAdamOpts), vp, vp]),
            "beta_relocate_workspace_bytes": (sz, [i32]),
            "beta_dssim_workspace_bytes": (sz, [C, i32]),
            "beta_l1_dssim_loss": (ctypes.c_int, [C, i32, vp, vp, ctypes.c_float, vp, vp, vp, sz, vp]),
            "beta_relocate": (ctypes.c_int, [i32, i32, i32, vp, vp, vp, vp, ctypes.c_float, vp, sz, vp, vp, vp]),
        }
        for name, (res, args) in sig.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
        return L


def check(fn: str, code: int):
    if code != BETA_OK:
        raise BetaError(fn, code, load().beta_status_string(code).decode())


def adam_default_opts(lr: dict | None = None, **kw) -> BetaAdamOpts:
    """The appendix hyperparameters; lr maps ADAM_GROUPS names to rates."""
    o = BetaAdamOpts()
    load().beta_adam_default_opts(ctypes.byref(o))
    for k, v in (lr or {}).items():
        o.lr[ADAM_GROUPS.index(k)] = v
    for k, v in kw.items():
        setattr(o, k, v)
    return o


def default_opts(**kw) -> BetaOpts:
    o = BetaOpts()
    load().beta_default_opts(ctypes.byref(o))
    for k, v in kw.items():
        setattr(o, k, v)
    return o


def make_cameras(cams) -> ctypes.Array:
    """scenes.Camera list -> BetaCamera[V] (host array)."""
    arr = (BetaCamera * len(cams))()
    for k, c in enumerate(cams):
        R = [float(x) for x in c.R.reshape(-1)]
        for j in range(9):
            arr[k].R[j] = R[j]
        for j in range(3):
            arr[k].t[j] = float(c.t[j])
            arr[k].bg[j] = float(c.bg[j])
        arr[k].fx, arr[k].fy, arr[k].cx, arr[k].cy = c.fx, c.fy, c.cx, c.cy
        arr[k].near_plane = c.near
        arr[k].width, arr[k].height = int(c.width), int(c.height)
    return arr


def make_params(n: int, pitch: int, n_lobes: int, ptr: int) -> BetaParams:
    p = BetaParams()
    p.n, p.pitch, p.n_lobes, p.reserved, p.planes = n, pitch, n_lobes, 0, ptr
    return p


def inf_opts() -> dict:
    return {"b_lo": -math.inf, "b_hi": math.inf}
