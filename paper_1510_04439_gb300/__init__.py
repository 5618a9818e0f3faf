"""GB300 (sm_103a) binned local linear FPCA smoother.

The compute path is libfpca.so (hand-written CUDA kernels behind the C ABI of
include/fpca.h); ``binding`` loads it with ctypes and ``pipeline`` strings the
ABI calls together.  Importing the package does not load the library.
"""
__all__ = ["binding", "pipeline", "build"]
