"""GB300 (sm_103a) implementation of the Exact Regularized Point Particle
two-way coupling step (Gualtieri, Picano, Sardina & Casciola).

The computation lives in the CUDA library ``liberpp.so`` behind the C ABI of
``include/erpp.h``; this package is its PyTorch binding.
"""

from ._lib import (FP32, FP64, FULL_FORCE, KAHAN, LAG, NORMALIZE, PIC,  # noqa: F401
                   POINT_GATHER, SELF_REMOVAL, ErppError, load)
from .erpp import (Batch, Context, Interpolate, ParticleState, ScatterSource,  # noqa: F401
                   StokesFluid, shared_add_rate)

__all__ = ["Batch", "Context", "StokesFluid", "ParticleState", "ScatterSource", "Interpolate", "ErppError", "load",
           "shared_add_rate",
           "FP32", "FP64", "NORMALIZE", "SELF_REMOVAL", "KAHAN", "PIC", "POINT_GATHER", "LAG", "FULL_FORCE"]
