"""GB300-native particle-mesh force evaluation and BullFrog integration
(arXiv:2510.05206, Sec. 2.4-2.7) behind the C ABI of include/pmgb.h.

Importing the package loads nothing; the CUDA library is loaded (and must
exist) when a handle is created.
"""
from .pm import PM, Config, workspace_bytes  # noqa: F401
