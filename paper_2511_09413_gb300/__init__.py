"""GB300-native rail-based kinetic Monte Carlo ion-migration sweep
(arXiv 2511.09413).

- ``kmc``: ctypes binding of the C ABI (include/kmc.h) over libkmc.so, the
  hand-written sm_103a CUDA kernels.
- ``workloads``: seeded synthetic devices and voltage protocols.
- ``build``: in-tree nvcc build of libkmc.so.

Importing the package loads nothing; ``kmc.load()`` (called by every binding
function) raises if libkmc.so is absent, so there is no silent fallback.
"""
__all__ = ["kmc", "workloads", "build"]
