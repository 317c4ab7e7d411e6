"""GB300-native convolution gridding (Winkel, Lenz & Floeer 2016, arXiv 1604.06667).

The compute path is the CUDA library behind the C ABI in include/cygrid_gb300.h;
this package is its thin Python binding.  Submodules load lazily so that
``import paper_1604_06667_gb300`` works on machines without a GPU.
"""
__all__ = ["Gridder", "ang2pix_ring", "unit_vectors", "build", "autograd", "mapmaking", "Batch"]


def __getattr__(name):
    if name in ("Gridder", "ang2pix_ring", "unit_vectors"):
        from . import gridder
        return getattr(gridder, name)
    if name == "Batch":
        from .batch import Batch
        return Batch
    if name in ("autograd", "mapmaking"):
        import importlib
        return importlib.import_module("." + name, __name__)
    if name == "build":
        from .build import build
        return build
    raise AttributeError(name)
