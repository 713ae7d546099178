"""GB300-native SLIM boundary-element solver: AIM + internal-problem system matvec and GMRES.

The compute path is the CUDA library `libbem_aim.so` (sources in csrc/, C ABI declared in
include/bem_aim.h); `api` is a thin ctypes binding. Importing this package does not load the
library; `api.lib()` does, and fails loudly when it is missing.
"""
__all__ = ["synth"]
