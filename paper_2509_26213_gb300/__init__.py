"""GB300 bricked multi-resolution volume raycaster (sm_103a CUDA behind a C ABI).

Hot path (Drees & Risse, "Palace", arXiv 2509.26213): per-pixel ray generation, page-table
lookup into a brick atlas, footprint LOD selection, trilinear sampling, 1D RGBA transfer
function, front-to-back compositing with early termination; the LOD box-downsample, the
brick-request queue with an LRU brick cache, and the adjoint (gradients with respect to the
transfer function and the voxels).

The compiled library ``libvolrc.so`` is required: importing :class:`Volume` without it
raises ImportError (there is no CPU fallback).
"""
from .build import build  # noqa: F401

__all__ = ["build", "Volume", "RaycastFn", "plan"]


def __getattr__(name):
    if name in ("Volume", "RaycastFn", "plan", "camera_struct", "params_struct"):
        from . import volume
        return getattr(volume, name)
    raise AttributeError(name)
