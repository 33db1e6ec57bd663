"""GB300-native optimiser of screen-space blue-noise samplers built from a rank-1 lattice with
per-pixel toroidal shifts (Belcour & Heitz, SIGGRAPH '21 Talks).

The computation lives in ``libbnsampler.so`` (CUDA, sm_103a), reached through the C ABI of
``include/bn_sampler.h``; this package only marshals arguments.
"""
from ._lib import (BN_MODE_CONCURRENT, BN_MODE_NONINTERACTING, BN_OBJECTIVE_BLUE,  # noqa: F401
                   BN_INTEGRANDS_GAUSSIAN, BN_INTEGRANDS_HEAVISIDE,
                   BN_OBJECTIVE_LITERAL, BN_SCHEDULE_AUTO, BN_SCHEDULE_PERSISTENT,
                   BN_SCHEDULE_PLAIN, BN_SCHEDULE_TENSOR, BnError, load)
from .sampler import Batch, Result, Sampler, Server, SweepStats  # noqa: F401
