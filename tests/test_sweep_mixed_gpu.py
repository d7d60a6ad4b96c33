"""Sweeps with the mixed-precision (tensor-core) sigma: FP64 Davidson
control, decimation and transformation, bf16-slice sigma products. The
energy of every step is the FP64 Rayleigh quotient of the converged vector,
so at full bond dimension it reproduces FCI to far better than the mixed
sigma's own relative error: the bar is 1e-6 Ha. The Davidson tolerance on
|r|^2 follows what each sigma can resolve: BF16X3 keeps 24 significant bits
(relative error ~6e-8, |r|^2 floor far below 1e-10), BF16X2 16 bits
(~1.5e-5, so |r|^2 of a vector of norm 1 with |H psi| ~ 10 cannot go much
below ~1e-8), FP16X2 22 bits (~2.4e-7, |r|^2 floor ~1e-11); 1e-10, 1e-8 and
1e-10 respectively. FP16X2 also meets the renormalized operators of real
sweeps, whose blocks span many orders of magnitude (per-block scales)."""

import json
import os

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

GOLD = os.path.join(os.path.dirname(__file__), "golden", "fci_energies.json")


@pytest.mark.parametrize("prec,tol", [("BF16X3", 1e-10), ("BF16X2", 1e-8), ("FP16X2", 1e-10)])
def test_config1_mixed_sweeps_within_1e6_of_fci(prec, tol):
    from paper_2103_09976_gb300 import capi
    from synth import random_integrals
    gold = json.load(open(GOLD))["cfg1"]["energy"]
    t, v = random_integrals(8, 0)
    ctx = capi.dmrg_create(device=0, seed=0, dav_max_iter=400, sigma_prec=getattr(capi, "DMRG_" + prec))
    try:
        capi.dmrg_build_blocks(ctx, t, v, 8, 8, 0, 256)
        e, _ = capi.dmrg_sweep(ctx, [256] * 4, tol)
        log = capi.dmrg_sweep_log(ctx)
    finally:
        capi.dmrg_destroy(ctx)
    assert np.all(np.abs(e - gold) < 1e-6), (e, gold)
    assert all(l["converged"] for l in log), [(l["site"], l["iters"]) for l in log if not l["converged"]]
