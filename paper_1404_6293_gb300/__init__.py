"""GB300 binned forward rasterizer: the AssignBin / Schedule / Process hot path
of the Piko raster pipeline (arXiv 1404.6293) as CUDA kernels for sm_103a
behind a C ABI (include/piko_raster.h).

Submodules: ``raster`` (Python API over the C ABI), ``scenes`` (seeded input
generators), ``build`` (nvcc build of the library).  Importing the package
does not load the CUDA library; constructing a ``Rasterizer`` does.
"""

__all__ = ["raster", "scenes", "build"]
