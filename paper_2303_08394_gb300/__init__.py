"""GB300-native Laplace kernel-independent FMM.

The hot path (V-list M2L and U-list P2P) and every other operator run in
hand-written sm_103a CUDA kernels inside ``libkifmm.so``, reached through
the C ABI in ``include/kifmm.h``.  This package only marshals arguments.
"""
from .fmm import FMMPlan, set_operator_cache  # noqa: F401
from . import _native  # noqa: F401
