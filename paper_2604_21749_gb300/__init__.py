"""GB300 visibility-buffer rasterizer (CuRast method, Schuetz et al. 2026).

Brute-force rasterization of massive indexed triangle meshes into a 64-bit
visibility buffer (28-bit depth, 36-bit global triangle id) by hand-written
CUDA kernels for sm_103a behind the C ABI of include/curast.h.  This package
is the Python binding of that library; importing it loads nothing until a
Renderer is created.
"""
from .build import build_library, lib_path  # noqa: F401


def __getattr__(name):
    if name in ("Renderer", "InterpolateFn", "CurastError", "Config", "Stats", "View", "load", "EXPORTS"):
        from . import api
        return getattr(api, name)
    raise AttributeError(name)
