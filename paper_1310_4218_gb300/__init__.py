"""GB300-native column-physics load balancing (over-decomposed VPs, on-device
load measurement, GreedyLB / RefineSwapLB / task-queue assignment).

The compute path is liblb.so (hand-written CUDA for sm_103a behind the C ABI
of include/lb.h); `lb` is its ctypes binding and `sim` allocates device
buffers with PyTorch.  Nothing here computes on the CPU.
"""
from . import lb
from .lb import LBError, load_library

__all__ = ["lb", "LBError", "load_library"]
