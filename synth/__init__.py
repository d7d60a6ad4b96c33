"""Seeded synthetic inputs shared by the oracle and the GPU library.

This package only draws numbers and shapes of workloads: integrals, sector
dimension lists, wavefunction vectors and serving request streams. It holds
none of the DMRG arithmetic (no operators, no sector bookkeeping, no sigma),
so that the oracle and the CUDA path can both consume its output without
sharing any of the method's code.
"""

from .integrals import random_integrals, femoco_like_integrals
from .sectors import gaussian_sector_dims, mirrored_sectors
from .vectors import random_unit_vector
from .requests import poisson_requests

__all__ = [
    "random_integrals",
    "femoco_like_integrals",
    "gaussian_sector_dims",
    "mirrored_sectors",
    "random_unit_vector",
    "poisson_requests",
]
