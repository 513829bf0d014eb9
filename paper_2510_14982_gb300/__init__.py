"""GB300-native Artificial Protozoa Optimizer (APO) population update.

The compute path is the C-ABI library ``libapo.so`` (hand-written sm_103a CUDA,
declared in ``include/apo.h``); :mod:`paper_2510_14982_gb300.apo` is its thin
ctypes binding.  Importing this package does not load the library; importing
:mod:`paper_2510_14982_gb300.apo` does, and fails loudly when it is missing.
"""
__all__ = ["apo", "inputs", "build"]
