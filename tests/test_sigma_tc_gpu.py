"""GPU parity of the mixed-precision sigma (bf16-slice products on tcgen05,
small classes on the CUDA cores) against the CPU oracle and against the FP64
GPU path, through the C ABI.

Tolerances follow from the arithmetic. BF16X3 represents every operand to
24 significant bits and drops slice products below 2^-24 relative. The
tensor cores accumulate in FP32, and their rounding error grows with the
number of main (hi x hi) MMAs in one accumulation: each such step can lose
up to about 2^-23 of the running value. The intermediate X = L psi is one
chain of m/16 main steps (m the psi block rows: up to 23 steps for the
355-row blocks below, about 2.7e-6); the sigma tile accumulation is cut
after at most 8 main steps and added into an FP32 running sum of the item
(one more rounding per flush group, about 1e-6). Measured: about 1e-6 at
blocks up to 107, 2.5e-6 at blocks up to 355: bar 5e-6 of max|sigma|. BF16X2 keeps 16 bits per operand (2^-17
representation error, dropped slice products ~2^-16): measured 6.6e-6, bar
2e-5. FP16X2 keeps 22 bits per operand (two fp16 slices of operands scaled
by powers of two, dropped lo x lo products ~2^-22) with the same bounded FP32
accumulation as BF16X3: bar 5e-6. Small classes (all blocks at most 32 wide)
run as FP32 products of at most 32 terms: about 1e-7.
"""

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

TOL = {1: 2e-5, 2: 5e-6, 3: 5e-6}


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


@pytest.mark.parametrize("prec", [2, 1, 3])
@pytest.mark.parametrize("M,nsp,ntot,seed", [
    (24, 3, 6, 1),        # tiny blocks: every class on the CUDA cores
    (120, 4, 8, 2),
    (1200, 3, 6, 3),      # blocks up to 107: several stage-1 stages, two 64-column halves
    (4000, 3, 6, 4),      # blocks up to 355: several 128-row / 128-column tiles, 3 psi chunks
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


@pytest.mark.parametrize("prec", [1, 3])
@pytest.mark.parametrize("M,nsp,ntot,seed", [(1200, 3, 6, 3), (4000, 3, 6, 4)])
def test_producer_settings_give_the_same_bits(capi, prec, M, nsp, ntot, seed):
    """One producer warp filling every ring stage and three warps filling one
    stage each move the same tiles into the same places: sigma is bitwise the
    same for both settings and for the plan's default, and within the bar
    against the oracle."""
    from synth import gaussian_sector_dims, mirrored_sectors, random_unit_vector
    left = gaussian_sector_dims(M, n_spatial=nsp, n_tot=ntot)
    right = mirrored_sectors(left, n_tot=ntot)
    nL, n = 2 * nsp, 4 * nsp
    ys, used = {}, {}
    for producers in (0, 1, 3):
        ctx = capi.dmrg_create(device=0, sigma_prec=prec, tc_producers=producers)
        try:
            capi.dmrg_load_synthetic(ctx, nL, n, ntot, 0, left, right, seed)
            size = capi.dmrg_psi_layout(ctx)["size"]
            x = random_unit_vector(size, seed + 10)
            y = np.zeros_like(x)
            capi.dmrg_sigma(ctx, -1, x, y)
            ys[producers] = y
            used[producers] = capi.dmrg_get_sigma_info(ctx)["tc_producers"]
        finally:
            capi.dmrg_destroy(ctx)
    assert used[1] == 1 and used[3] == 3 and used[0] in (1, 3)
    assert np.array_equal(ys[1], ys[3]) and np.array_equal(ys[0], ys[1])
    ref = _oracle_full(left, right, nL, n, (ntot, 0), seed, x)
    assert np.abs(ys[3] - ref).max() / np.abs(ref).max() <= TOL[prec]


def test_sigma_tc_middle_bond_m2000_vs_fp64(capi):
    """K=108 (54|54), N=30, M=2000: BF16X3, BF16X2 and FP16X2 against the
    FP64 GPU path on the same context, plus the Rayleigh-quotient
    difference."""
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
        for prec in (2, 1, 3):
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


@pytest.mark.parametrize("factor", [1e-30, 1.0, 3e25])
def test_fp16x2_psi_scale_is_exact(capi, factor):
    """FP16X2 scales psi by a power of two from its largest element before the
    fp16 split: sigma(a psi) = a sigma(psi) to the FP16X2 bar for psi far
    outside the fp16 range, an all-zero psi gives exactly zero, and switching
    between the fp16 and the bf16 split on one context keeps both results."""
    from synth import gaussian_sector_dims, mirrored_sectors, random_unit_vector
    left = gaussian_sector_dims(1200, n_spatial=3, n_tot=6)
    right = mirrored_sectors(left, n_tot=6)
    ctx = capi.dmrg_create(device=0)
    try:
        capi.dmrg_load_synthetic(ctx, 6, 12, 6, 0, left, right, 3)
        size = capi.dmrg_psi_layout(ctx)["size"]
        x = random_unit_vector(size, 13)
        y64 = np.zeros_like(x)
        capi.dmrg_sigma(ctx, -1, x, y64)
        capi.dmrg_set_precision(ctx, 3)
        y = np.zeros_like(x)
        capi.dmrg_sigma(ctx, -1, x * factor, y)
        z = np.ones_like(x)
        capi.dmrg_sigma(ctx, -1, np.zeros_like(x), z)
        capi.dmrg_set_precision(ctx, 2)
        yb = np.zeros_like(x)
        capi.dmrg_sigma(ctx, -1, x, yb)
        capi.dmrg_set_precision(ctx, 3)
        y2 = np.zeros_like(x)
        capi.dmrg_sigma(ctx, -1, x * factor, y2)
    finally:
        capi.dmrg_destroy(ctx)
    assert np.all(np.isfinite(y))
    assert np.abs(y / factor - y64).max() <= TOL[3] * np.abs(y64).max()
    assert np.abs(yb - y64).max() <= TOL[2] * np.abs(y64).max()
    assert np.array_equal(y, y2)
    assert not z.any()
