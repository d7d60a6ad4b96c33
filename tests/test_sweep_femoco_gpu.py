"""Sweeps on FeMoco-shaped integrals (couplings decaying as exp(-|p-q|/8),
N/K = 113/76, odd 2Sz) at reduced size: K=8, N=11, 2Sz=1, M=32 < full.

FP64 sweeps follow the oracle's plain DMRG step by step (energies to
1e-9 Ha, as in test_sweep_gpu). Sweeps with the BF16X3 sigma keep FP64
Davidson control, decimation and transformation; their eigenvectors carry
the mixed sigma's ~1e-5 relative error into each truncation, so the kept
bases differ from the FP64 run at that order and the swept energies at
about the square of it times the energy scale: the bar is 1e-6 Ha."""

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

K, N, TWO_SZ, M = 8, 11, 1, 32


def _gpu(prec):
    from paper_2103_09976_gb300 import capi
    from synth.integrals import femoco_like_integrals
    t, v = femoco_like_integrals(K=K, seed=2)
    ctx = capi.dmrg_create(device=0, seed=2, dav_max_iter=400, sigma_prec=getattr(capi, "DMRG_" + prec))
    try:
        capi.dmrg_build_blocks(ctx, t, v, K, N, TWO_SZ, M)
        e, d = capi.dmrg_sweep(ctx, [M, M], 1e-20 if prec == "FP64" else 1e-12)
        log = capi.dmrg_sweep_log(ctx)
    finally:
        capi.dmrg_destroy(ctx)
    return e, d, log


def test_fp64_sweeps_follow_oracle():
    from oracle.dmrg import PlainDMRG
    from synth.integrals import femoco_like_integrals
    t, v = femoco_like_integrals(K=K, seed=2)
    ora = PlainDMRG(t, v, N, TWO_SZ, seed=2, dav_tol=1e-20, dav_max_iter=400)
    ora.build_blocks(M)
    e_ref, d_ref = ora.sweep([M, M])
    e, d, log = _gpu("FP64")
    assert len(log) == len(ora.log)
    for g, o in zip(log, ora.log):
        assert (g["site"], g["psi_size"]) == (o["i"], o["dim"])
        assert abs(g["energy"] - o["energy"]) < 1e-9, (g, o)
    assert np.all(np.abs(e - np.array(e_ref)) < 1e-9)


def test_mixed_sweeps_match_fp64_sweeps():
    e64, _, _ = _gpu("FP64")
    e16, _, log = _gpu("BF16X3")
    assert all(l["converged"] for l in log)
    assert np.all(np.abs(e16 - e64) < 1e-6), (e16, e64)
