"""GPU parity of the tensor-core sigma (bf16-slice products, tcgen05) against
the CPU oracle and against the FP64 GPU path, through the C ABI.

Tolerances follow from the arithmetic. BF16X3 represents every operand to
24 significant bits and drops slice products below 2^-24 relative, so the
products themselves are good to a few 2^-24. The tensor cores accumulate in
FP32: an output element of one segment (at most 32 tasks, then added in
FP64) receives n ~ 6 x K x 32 rounded additions (K up to 355 here), so its
rounding error is about 2^-24 sqrt(n) ~ 3e-6 of the magnitudes entering it,
with a tail up to ~10x that over 1e5-1e6 outputs: bar 5e-5 of max|sigma|.
BF16X2 keeps 16 bits (2^-17 representation error, dropped products ~2^-16):
bar 2e-3.
"""

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

TOL = {1: 2e-3, 2: 5e-5}


@pytest.fixture(scope="module")
def capi():
    from paper_2103_09976_gb300 import capi as c
    return c


def _oracle_full(left, right, nL, n, Q, seed, x):
    from oracle.nc import nc_terms
    from oracle.sigma import psi_layout, sigma_blocks, synthetic_ops
    bL, bR, oL, oR, _ = synthetic_ops(left, right, nL, n, seed=seed)
    lay, size = psi_layout(bL, bR, Q)
    return sigma_blocks(x, lay, nc_terms(nL, n), oL, oR)


@pytest.mark.parametrize("prec", [2, 1])
@pytest.mark.parametrize("M,nsp,ntot,seed", [
    (24, 3, 6, 1),        # tiny blocks: most of every 128-row tile is padding
    (120, 4, 8, 2),
    (1200, 3, 6, 3),      # blocks up to 107: several K1 stages, two 64-column X sub-chunks
    (4000, 3, 6, 4),      # blocks up to 355: several 128-row / 128-column tiles, 3 X passes
])
def test_sigma_tc_matches_oracle(capi, prec, M, nsp, ntot, seed):
    from synth import gaussian_sector_dims, mirrored_sectors, random_unit_vector
    left = gaussian_sector_dims(M, n_spatial=nsp, n_tot=ntot)
    right = mirrored_sectors(left, n_tot=ntot)
    nL, n = 2 * nsp, 4 * nsp
    ctx = capi.dmrg_create(device=0, sigma_prec=prec)
    try:
        capi.dmrg_load_synthetic(ctx, nL, n, ntot, 0, left, right, seed)
        size = capi.dmrg_psi_layout(ctx)["size"]
        x = random_unit_vector(size, seed + 10)
        y = np.zeros_like(x)
        capi.dmrg_sigma(ctx, -1, x, y)
        y2 = np.zeros_like(x)
        capi.dmrg_sigma(ctx, -1, x, y2)
    finally:
        capi.dmrg_destroy(ctx)
    ref = _oracle_full(left, right, nL, n, (ntot, 0), seed, x)
    err = np.abs(y - ref).max() / np.abs(ref).max()
    assert err <= TOL[prec], err
    assert np.array_equal(y, y2), "tensor-core sigma must be bitwise deterministic"


def test_sigma_tc_middle_bond_m2000_vs_fp64(capi):
    """K=108 (54|54), N=30, M=2000: BF16X3 and BF16X2 against the FP64 GPU
    path on the same context, plus the Rayleigh-quotient difference."""
    from synth import gaussian_sector_dims, mirrored_sectors, random_unit_vector
    left = gaussian_sector_dims(2000)
    right = mirrored_sectors(left)
    ctx = capi.dmrg_create(device=0)
    try:
        capi.dmrg_load_synthetic(ctx, 108, 216, 30, 0, left, right, 1)
        size = capi.dmrg_psi_layout(ctx)["size"]
        x = random_unit_vector(size, 1)
        y64 = np.zeros_like(x)
        capi.dmrg_sigma(ctx, -1, x, y64)
        out = {}
        for prec in (2, 1):
            capi.dmrg_set_precision(ctx, prec)
            y = np.zeros_like(x)
            capi.dmrg_sigma(ctx, -1, x, y)
            out[prec] = y
    finally:
        capi.dmrg_destroy(ctx)
    for prec, y in out.items():
        err = np.abs(y - y64).max() / np.abs(y64).max()
        assert err <= TOL[prec], (prec, err)
        rq = abs(x @ y - x @ y64) / abs(x @ y64)
        assert rq <= TOL[prec], (prec, rq)
