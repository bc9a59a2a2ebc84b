"""GB300 (sm_103a) hybrid sparse eigensolver: the C-ABI library libeig.so and its thin binding.

Every arithmetic step runs in the library's CUDA kernels; this package only marshals
arguments (see binding.py).  There is no CPU fallback: without the built library or a
CUDA device the binding raises.
"""
__all__ = ["binding"]
