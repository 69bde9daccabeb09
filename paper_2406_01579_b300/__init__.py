"""B300-native tetrahedron splatting rasterizer (TeT-Splatting, Sec. 3.2-3.3,
App. A): CUDA kernels for sm_103a behind the C ABI of include/tets.h, with a
thin PyTorch binding.  There is no CPU fallback: importing the rasterizer
requires the built libtets.so."""

from . import camera  # noqa: F401
from ._lib import TetsError, load  # noqa: F401
from .rasterizer import (Params, Rasterizer, SceneTensors, TetRender, TetRenderBatch,  # noqa: F401
                         fit_grid, make_camera, render)

__all__ = ["Params", "Rasterizer", "SceneTensors", "TetRender", "TetRenderBatch", "render",
           "make_camera", "load", "TetsError", "camera", "fit_grid"]
