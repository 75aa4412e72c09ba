"""GB300-native octree-block multigrid (arXiv 2403.08063): CUDA kernels for sm_103a behind a C ABI.

The solver lives in libocmg.so (include/octmg.h); this package is its thin Python front end.
"""
from ._lib import MGError, load  # noqa: F401
from .api import Batch, Forest, MGSolveFn, alu_peaks  # noqa: F401
