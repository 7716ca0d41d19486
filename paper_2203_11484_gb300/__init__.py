"""GB300 (sm_103a) implementation of the hybrid close-range VPL method of
Jin, Wang, Zheng, Hua and Huo (arXiv 2203.11484): patch-based VPLs on the
close range picked out by the camera, sparse instant radiosity for the
distant part, and the per-pixel indirect gather with BVH shadow rays.

The compute path is libvpl.so (hand-written CUDA behind the C ABI of
include/vpl.h); ``vpl`` is its Python binding and ``workloads`` the seeded
synthetic inputs.
"""
from . import workloads  # noqa: F401

__all__ = ["workloads", "vpl", "build"]
