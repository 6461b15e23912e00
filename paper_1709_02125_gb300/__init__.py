"""GB300-native out-of-core executor for stencil loop chains (arXiv 1709.02125).

`oc` is the ctypes binding of liboc.so (C ABI in include/oc.h); `_build` compiles it
for sm_103a. Nothing in this package computes a loop on the CPU.
"""
from . import oc  # noqa: F401
from .oc import Executor, load, run_chain  # noqa: F401
