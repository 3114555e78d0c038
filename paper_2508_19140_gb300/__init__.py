"""GB300-native (sm_103a) tiled point rasterizer of INPC's "bag of tricks"
(arXiv 2508.19140): projection, split radix sort by (tile, depth, index),
front-to-back blending (Eq. 1) and the corrected backward pass (Eq. 2),
behind the C ABI of include/inpc_rast.h.

Submodules: ``build`` (compiles the CUDA library in-tree), ``rast`` (ctypes
binding and autograd), ``scenes`` (seeded synthetic workloads). Importing the
package does not load the CUDA library; the first compute call does, and
fails loudly if it has not been built.
"""
__all__ = ["build", "rast", "scenes"]
