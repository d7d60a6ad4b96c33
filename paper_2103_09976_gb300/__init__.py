"""GB300-native two-site ab initio DMRG hot path (sigma = H_eff . psi).

The computation lives in libdmrg.so (CUDA, sm_103a) behind the C ABI of
include/dmrg.h; `capi` is a thin ctypes binding with the same names.
"""

from . import capi  # noqa: F401
