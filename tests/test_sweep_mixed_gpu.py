"""Sweeps with the mixed-precision (tensor-core) sigma: FP64 Davidson
control, decimation and transformation, bf16-slice sigma products. The
energy of every step is the FP64 Rayleigh quotient of the converged vector,
so at full bond dimension it reproduces FCI to far better than the mixed
sigma's own relative error (about 1e-5): the bar is 1e-6 Ha."""

import json
import os

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

GOLD = os.path.join(os.path.dirname(__file__), "golden", "fci_energies.json")


@pytest.mark.parametrize("prec", ["BF16X3", "BF16X2"])
def test_config1_mixed_sweeps_within_1e6_of_fci(prec):
    from paper_2103_09976_gb300 import capi
    from synth import random_integrals
    gold = json.load(open(GOLD))["cfg1"]["energy"]
    t, v = random_integrals(8, 0)
    ctx = capi.dmrg_create(device=0, seed=0, dav_max_iter=400, sigma_prec=getattr(capi, "DMRG_" + prec))
    try:
        capi.dmrg_build_blocks(ctx, t, v, 8, 8, 0, 256)
        e, _ = capi.dmrg_sweep(ctx, [256] * 4, 1e-10)
        log = capi.dmrg_sweep_log(ctx)
    finally:
        capi.dmrg_destroy(ctx)
    assert np.all(np.abs(e - gold) < 1e-6), (e, gold)
    assert all(l["converged"] for l in log)
