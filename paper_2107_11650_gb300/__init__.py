"""GB300-native separable low-rank Hankel MRI reconstruction (SHLR family).

The compute path is the C-ABI library ``libselr.so`` (hand-written sm_103a
CUDA kernels, declared in ``include/selr.h``).  ``api`` wraps it with the
same entry-point names for callers holding torch CUDA tensors.
"""
from .build import build  # noqa: F401

__all__ = ["build"]
