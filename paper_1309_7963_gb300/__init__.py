"""pnuc: GB300-native event-parallel Monte Carlo of non-elastic proton-nucleus interactions
(20-250 MeV): intranuclear cascade + evaporation after arXiv:1309.7963.

The work runs in libpnuc (CUDA, sm_103a) behind the C ABI of include/pnuc.h; `pnuc` is its
Python binding and `inputs` the seeded synthetic workloads.
"""
from . import inputs  # noqa: F401
from .pnuc import (COUNTER_NAMES, FLAGS, RESIDUAL_DTYPE, SECONDARY_DTYPE, Context, PnucError,  # noqa: F401
                   load, sort_secondaries)
