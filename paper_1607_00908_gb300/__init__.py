"""GB300-native detection of topological changes in dynamic Voronoi diagrams.

The hot path (threshold, periodic labelling, 1/1024-site centroids, exact
digital Voronoi owners, Delaunay links, frame-to-frame isomorphism and
breaking/arising links) runs in hand-written sm_103a CUDA kernels behind the
C ABI of ``include/vd.h`` (libvd.so). ``vd`` is the ctypes binding,
``inputs`` the seeded synthetic workloads, ``build`` the in-tree nvcc build.
"""
from . import inputs  # noqa: F401

__all__ = ["inputs", "vd", "build"]
