"""GPU parity of sigma = H_eff . psi (FP64) against the CPU oracle, through the C ABI.

Tolerance (FP64): both sides sum the same products in different orders; the
rounding error of a sum of n random-sign products grows like sqrt(n) ulps
of the partial sums, which for the ~1e8-1e9 products per element at the
middle bond stays below 1e-13 of max|sigma|. The bar is 1e-12 of max|sigma|
elementwise - a dropped term, a sign or a transposed operand changes sigma
at the 1e-3 level or more.
"""

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

TOL = 1e-12


@pytest.fixture(scope="module")
def capi():
    from paper_2103_09976_gb300 import capi as c
    return c


def _oracle_full(left, right, nL, n, Q, seed, x):
    from oracle.nc import nc_terms
    from oracle.sigma import psi_layout, sigma_blocks, synthetic_ops
    bL, bR, oL, oR, _ = synthetic_ops(left, right, nL, n, seed=seed)
    lay, size = psi_layout(bL, bR, Q)
    return sigma_blocks(x, lay, nc_terms(nL, n), oL, oR), lay


def _layout_matches(lay_gpu, lay_oracle):
    assert len(lay_gpu["m_l"]) == len(lay_oracle)
    for k, (qL, qR, mL, mR, off) in enumerate(lay_oracle):
        assert tuple(lay_gpu["q_l"][k]) == qL
        assert lay_gpu["m_l"][k] == mL and lay_gpu["m_r"][k] == mR and lay_gpu["offset"][k] == off


@pytest.mark.parametrize("M,nsp,ntot,seed", [
    (24, 3, 6, 1),        # tiny: single tile per block
    (120, 4, 8, 2),       # 25 sectors, blocks up to 9
    (1200, 3, 6, 3),      # blocks up to 107: several 32-row tiles and 64-column chunks, ragged tails
    (4000, 3, 6, 4),      # blocks up to 355: several 256-column tiles
])
def test_sigma_fp64_matches_oracle(capi, M, nsp, ntot, seed):
    from synth import gaussian_sector_dims, mirrored_sectors, random_unit_vector
    left = gaussian_sector_dims(M, n_spatial=nsp, n_tot=ntot)
    right = mirrored_sectors(left, n_tot=ntot)
    nL, n = 2 * nsp, 4 * nsp
    ctx = capi.dmrg_create(device=0)
    try:
        capi.dmrg_load_synthetic(ctx, nL, n, ntot, 0, left, right, seed)
        lay = capi.dmrg_psi_layout(ctx)
        x = random_unit_vector(lay["size"], seed + 10)
        y = np.zeros_like(x)
        capi.dmrg_sigma(ctx, -1, x, y)
        y2 = np.zeros_like(x)
        capi.dmrg_sigma(ctx, -1, x, y2)
    finally:
        capi.dmrg_destroy(ctx)
    ref, olay = _oracle_full(left, right, nL, n, (ntot, 0), seed, x)
    _layout_matches(lay, olay)
    scale = np.abs(ref).max()
    assert np.abs(y - ref).max() <= TOL * scale
    assert np.array_equal(y, y2), "sigma must be bitwise deterministic"


def test_sigma_device_pointers_equal_host_pointers(capi):
    import torch
    from synth import gaussian_sector_dims, mirrored_sectors, random_unit_vector
    left = gaussian_sector_dims(200, n_spatial=4, n_tot=8)
    right = mirrored_sectors(left, n_tot=8)
    ctx = capi.dmrg_create(device=0)
    try:
        capi.dmrg_load_synthetic(ctx, 8, 16, 8, 0, left, right, 7)
        n = capi.dmrg_psi_layout(ctx)["size"]
        x = random_unit_vector(n, 1)
        yh = np.zeros(n)
        capi.dmrg_sigma(ctx, -1, x, yh)
        xd = torch.from_numpy(x).cuda()
        yd = torch.zeros(n, dtype=torch.float64, device="cuda")
        capi.dmrg_sigma(ctx, -1, xd, yd)
        torch.cuda.synchronize()
    finally:
        capi.dmrg_destroy(ctx)
    assert np.array_equal(yh, yd.cpu().numpy())


def test_sigma_empty_output_blocks_and_single_sector(capi):
    """Degenerate layouts: one sector per side; sectors that no operator reaches."""
    from synth import random_unit_vector
    from oracle.nc import nc_terms
    from oracle.sigma import psi_layout, sigma_blocks, synthetic_ops
    for left, right in (([(3, 1, 5)], [(3, -1, 4)]),
                        ([(0, 0, 1), (2, 0, 3), (4, 0, 2)], [(2, 0, 2), (4, 0, 3), (6, 0, 1)])):
        ctx = capi.dmrg_create(device=0)
        try:
            capi.dmrg_load_synthetic(ctx, 8, 16, 6, 0, left, right, 3)
            n = capi.dmrg_psi_layout(ctx)["size"]
            x = random_unit_vector(n, 4)
            y = np.full(n, np.nan)
            capi.dmrg_sigma(ctx, -1, x, y)
        finally:
            capi.dmrg_destroy(ctx)
        bL, bR, oL, oR, _ = synthetic_ops(left, right, 8, 16, seed=3)
        lay, size = psi_layout(bL, bR, (6, 0))
        ref = sigma_blocks(x, lay, nc_terms(8, 16), oL, oR)
        assert np.all(np.isfinite(y))
        assert np.abs(y - ref).max() <= TOL * max(1.0, np.abs(ref).max())


def test_invalid_inputs_rejected(capi):
    ctx = capi.dmrg_create(device=0)
    try:
        with pytest.raises(capi.DMRGError) as e:  # unsorted sectors
            capi.dmrg_load_synthetic(ctx, 8, 16, 8, 0, [(4, 0, 2), (3, 1, 2)], [(4, 0, 2)], 1)
        assert e.value.status == capi.DMRG_EINVAL
        with pytest.raises(capi.DMRGError) as e:  # 2Sz parity
            capi.dmrg_load_synthetic(ctx, 8, 16, 8, 0, [(4, 1, 2)], [(4, 0, 2)], 1)
        assert e.value.status == capi.DMRG_EINVAL
        with pytest.raises(capi.DMRGError) as e:  # nothing loaded
            capi.dmrg_sigma(ctx, -1, np.zeros(4), np.zeros(4))
        assert e.value.status == capi.DMRG_ESTATE
        capi.dmrg_load_synthetic(ctx, 8, 16, 8, 0, [(4, 0, 2)], [(4, 0, 2)], 1)
        with pytest.raises(capi.DMRGError) as e:  # NULL pointer
            capi.dmrg_sigma(ctx, -1, None, np.zeros(4))
        assert e.value.status == capi.DMRG_EINVAL
        buf = np.zeros(8)
        with pytest.raises(capi.DMRGError):  # overlapping psi / sigma
            capi.dmrg_sigma(ctx, -1, buf, buf[2:])
    finally:
        capi.dmrg_destroy(ctx)


@pytest.mark.parametrize("M,size,nblk", [(2000, 106004, 104), (4000, 424716, 116), (6000, 956036, 120)])
def test_sigma_middle_bond_sampled_blocks(capi, M, size, nblk):
    """K=108 (54|54), N=30, Sz=0 at the benchmark's bond dimensions: checked on
    3x3 sampled entries of three output blocks (largest, median, smallest).
    At M=2000 the work list is autotuned first, as bench.py times it."""
    from synth import gaussian_sector_dims, mirrored_sectors, random_unit_vector
    from oracle.sigma import synthetic_sigma_sampled
    left = gaussian_sector_dims(M)
    right = mirrored_sectors(left)
    ctx = capi.dmrg_create(device=0)
    try:
        capi.dmrg_load_synthetic(ctx, 108, 216, 30, 0, left, right, 1)
        if M == 2000:
            capi.dmrg_autotune(ctx, -1)
        lay = capi.dmrg_psi_layout(ctx)
        info = capi.dmrg_get_sigma_info(ctx)
        x = random_unit_vector(lay["size"], 1)
        y = np.zeros_like(x)
        capi.dmrg_sigma(ctx, -1, x, y)
    finally:
        capi.dmrg_destroy(ctx)
    assert lay["size"] == size and len(lay["m_l"]) == nblk
    assert info["n_terms"] == 23654
    if M == 2000:
        assert info["op_elements"] == 2130976408
        assert abs(info["flops"] - 0.568442744e12) < 1e3
    order = np.argsort(lay["m_l"] * lay["m_r"])
    pick = [order[-1], order[len(order) // 2], order[0]]
    samples = []
    for k in pick:
        ml, mr = int(lay["m_l"][k]), int(lay["m_r"][k])
        samples.append((tuple(lay["q_l"][k]), np.unique([0, ml // 2, ml - 1]),
                        np.unique([0, mr // 3, mr - 1])))
    ref = synthetic_sigma_sampled(left, right, 108, 216, 1, (30, 0), x, samples)
    for k, (q, rows, cols) in zip(pick, samples):
        off, ml, mr = lay["offset"][k], lay["m_l"][k], lay["m_r"][k]
        got = y[off:off + ml * mr].reshape(ml, mr)[np.ix_(rows, cols)]
        scale = max(np.abs(ref[q]).max(), 1e-300)
        assert np.abs(got - ref[q]).max() <= TOL * scale, q
