"""GB300-native solver for the MPFC convex-splitting schemes (arXiv:1208.2643).

The compute path is libmpfc (hand-written CUDA for sm_103a behind the C ABI of
include/mpfc.h); ``mpfc`` is its Python binding and ``inputs`` builds seeded
initial data.  Importing the package does not load the CUDA library.
"""
__all__ = ["mpfc", "inputs", "build"]
