"""GB300-native oracles for a neural-network constraint y = NN(x) inside an interior-point method.

The compute path is libnnc.so (CUDA for sm_103a, C ABI in include/nnc.h); `nnc` is its ctypes
binding.  Build the library with `paper_2509_22462_gb300.build.build()`.
"""
from . import nnc  # noqa: F401
from .nnc import Net, NNCError, eval_batched, load_library, launch_count  # noqa: F401
