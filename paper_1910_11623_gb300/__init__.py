"""GB300-native hot path of the deep FBSDE solver of arXiv 1910.11623.

The compute lives in libfbsde.so (C ABI, include/fbsde.h): Philox noise,
Euler-Maruyama paths, the network u(t, x; Theta) and Z = grad_x u, the loss
and its Theta-gradient, and Adam.  This package only marshals arguments
(`_lib`, same names as the C entry points) and manages torch-owned buffers
(`solver`).
"""
from .solver import ArchSpec, Group, ProblemSpec, RolloutLoss, Solver, TrainGraph, param_count, philox4x32_10  # noqa: F401
from . import workloads  # noqa: F401
