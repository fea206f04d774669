"""GB300 (sm_103a) Beta-splatting rasterizer: the data-parallel hot path of
Deformable Beta Splatting (arXiv 2501.18630).

  scenes     seeded synthetic scenes and cameras (inputs only)
  _lib       ctypes binding of libbetasplat.so (include/beta_splat.h)
  render     device buffers, the four-step path, torch.autograd.Function
"""
__all__ = ["scenes", "build_library", "load_library"]


def build_library(force: bool = False, verbose: bool = False) -> str:
    from .build import build
    return build(force=force, verbose=verbose)


def load_library():
    from . import _lib
    return _lib.load()
