"""GB300 (sm_103a) slice-and-store state-vector simulator for random Sycamore-pattern circuits,
after Pednault et al., arXiv:1910.09534.

The compute path is the native library ``_build/libsycsim.so`` (CUDA kernels + C ABI declared in
``include/sycsim.h``); ``_native`` is its ctypes binding with the same function names.
"""
from ._native import *  # noqa: F401,F403
from ._native import SimError, lib, gates_array, pinned_array  # noqa: F401
