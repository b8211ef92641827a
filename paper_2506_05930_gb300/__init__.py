"""GB300-native neural visibility cache hot path (Bokshansky & Meister,
"Neural Visibility Cache for Real-Time Light Sampling", JCGT 2025).

The compute lives in libnvc.so (hand-written CUDA for sm_103a behind the C
ABI of include/nvc.h); ``nvc`` is the Python binding with the same entry
point names, ``autograd`` puts the hand-written adjoint behind a
torch.autograd.Function, and ``examples`` holds runnable workloads.
"""
from .build import build, LIB  # noqa: F401

__all__ = ["build", "LIB"]
