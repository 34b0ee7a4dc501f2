"""GB300 (sm_103a) implementation of the Exact Regularized Point Particle
two-way coupling step (Gualtieri, Picano, Sardina & Casciola).

The computation lives in the CUDA library ``liberpp.so`` behind the C ABI of
``include/erpp.h``; this package is its PyTorch binding.
"""

from ._lib import FP32, FP64, KAHAN, NORMALIZE, SELF_REMOVAL, ErppError, load  # noqa: F401
from .erpp import Context, ParticleState  # noqa: F401

__all__ = ["Context", "ParticleState", "ErppError", "load", "FP32", "FP64", "NORMALIZE",
           "SELF_REMOVAL", "KAHAN"]
