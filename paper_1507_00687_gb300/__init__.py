"""GB300 (sm_103a) recursive fast matrix multiplication with power-of-two
diagonal scaling, after Ballard, Benson, Druinsky, Lipshitz and Schwartz,
"Improving the numerical stability of fast matrix multiplication".

The compute path is libfmm.so (CUDA kernels behind the C ABI of
include/fmm.h); this package adds a ctypes binding, the built-in rules and
PyTorch wrappers.  ``import paper_1507_00687_gb300.api`` requires the built
library and raises otherwise.
"""
__all__ = ["api", "rules", "inputs", "build"]
