"""GB300-native coupled cluster Monte Carlo time step.

The computation lives in the CUDA library built from ``csrc/`` (C ABI in
``include/ccmc.h``); ``ccmc`` is its ctypes binding.
"""
from .ccmc import Batch, CCMCError, Context, colocation, from_workload, load  # noqa: F401

__all__ = ["Batch", "CCMCError", "Context", "colocation", "from_workload", "load"]
