"""GB300-native Barnes-Hut octree treecode for Monte Carlo of charged systems.

The compute path is the CUDA library ``libbhmc.so`` (sources in ``csrc/``,
C-ABI in ``include/bhmc.h``); ``bhmc`` is its ctypes binding.  Importing the
package loads nothing: the library is opened on first use and a missing
library is an error, never a fallback.
"""
from . import workloads  # noqa: F401

__all__ = ["workloads"]
