"""GB300-native Monte Carlo Heston pricing with pathwise Greeks (arXiv 2309.10477).

The compute path is the CUDA library ``libhestonmc.so`` (C ABI in
``include/heston_mc.h``); ``native`` is its ctypes binding, ``workloads``
holds the seeded synthetic inputs.  Build with ``build.build()``.
"""
from . import native, workloads  # noqa: F401

__all__ = ["native", "workloads"]
