"""GB300 (sm_103a) swap-sweep library for the SMC-X method.

The compute path is the C-ABI shared library built from ``csrc/`` (CUDA
kernels for sm_103a behind ``include/smcx.h``).  ``smcx`` is its thin Python
binding; importing this package does not load the library until a binding
function is first used.
"""
__all__ = ["smcx", "inputs"]
