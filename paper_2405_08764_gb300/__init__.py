"""GB300-native patch dynamics for heterogeneous 2D convection-diffusion-reaction
problems in orthogonal curvilinear coordinates (arXiv 2405.08764).

The compute path is libpd.so (hand-written sm_103a CUDA behind the C ABI in
include/pd.h); this package holds its ctypes binding, the build script and the
seeded workload definitions.
"""
from . import workloads  # noqa: F401

__all__ = ["workloads", "Grid", "build"]


def __getattr__(name):
    if name == "Grid":
        from .api import Grid
        return Grid
    if name == "build":
        from .build import build
        return build
    raise AttributeError(name)
