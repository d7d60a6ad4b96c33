"""GPU sub-Hamiltonian parts of sigma (dmrg_sigma_part) against the
oracle's parts, and their sum against the full GPU sigma (FP64, 1e-12 of
max|sigma| as in test_sigma_gpu)."""

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("M,nsp,ntot,seed,P", [(120, 4, 8, 2, 3), (1200, 3, 6, 3, 4)])
def test_parts_match_oracle_and_sum_to_sigma(M, nsp, ntot, seed, P):
    from oracle.nc import nc_terms
    from oracle.sigma import psi_layout, sigma_part, synthetic_ops
    from paper_2103_09976_gb300 import capi
    from synth import gaussian_sector_dims, mirrored_sectors, random_unit_vector
    left = gaussian_sector_dims(M, n_spatial=nsp, n_tot=ntot)
    right = mirrored_sectors(left, n_tot=ntot)
    nL, n = 2 * nsp, 4 * nsp
    ctx = capi.dmrg_create(device=0)
    try:
        capi.dmrg_load_synthetic(ctx, nL, n, ntot, 0, left, right, seed)
        size = capi.dmrg_psi_layout(ctx)["size"]
        x = random_unit_vector(size, seed + 10)
        full = np.zeros(size)
        capi.dmrg_sigma(ctx, -1, x, full)
        parts = []
        for r in range(P):
            y = np.zeros(size)
            capi.dmrg_sigma_part(ctx, -1, r, P, x, y)
            parts.append(y)
        with pytest.raises(capi.DMRGError):
            capi.dmrg_sigma_part(ctx, -1, P, P, x, np.zeros(size))
    finally:
        capi.dmrg_destroy(ctx)
    bL, bR, oL, oR, _ = synthetic_ops(left, right, nL, n, seed=seed)
    lay, _ = psi_layout(bL, bR, (ntot, 0))
    terms = nc_terms(nL, n)
    scale = np.abs(full).max()
    for r in range(P):
        ref = sigma_part(x, lay, terms, oL, oR, r, P)
        assert np.abs(parts[r] - ref).max() <= 1e-12 * scale, r
    assert np.abs(sum(parts) - full).max() <= 1e-12 * scale


@pytest.mark.parametrize("M,nsp,ntot,seed,P", [(120, 4, 8, 2, 2), (1200, 3, 6, 3, 3)])
def test_partitioned_store_parts_sum_to_sigma(M, nsp, ntot, seed, P):
    """dmrg_load_synthetic_part: each rank's context stores only its
    sub-Hamiltonian's operators (together exactly the full store, each about
    1/P of it); its dmrg_sigma is the oracle's part, and the parts add up to
    the full sigma."""
    from oracle.nc import nc_terms
    from oracle.sigma import psi_layout, sigma_part, synthetic_ops
    from paper_2103_09976_gb300 import capi
    from synth import gaussian_sector_dims, mirrored_sectors, random_unit_vector
    left = gaussian_sector_dims(M, n_spatial=nsp, n_tot=ntot)
    right = mirrored_sectors(left, n_tot=ntot)
    nL, n = 2 * nsp, 4 * nsp
    ctx = capi.dmrg_create(device=0)
    try:
        capi.dmrg_load_synthetic(ctx, nL, n, ntot, 0, left, right, seed)
        size = capi.dmrg_psi_layout(ctx)["size"]
        total = capi.dmrg_get_sigma_info(ctx)["op_elements"]
        x = random_unit_vector(size, seed + 10)
        full = np.zeros(size)
        capi.dmrg_sigma(ctx, -1, x, full)
    finally:
        capi.dmrg_destroy(ctx)
    parts, elems = [], []
    for r in range(P):
        ctx = capi.dmrg_create(device=0)
        try:
            capi.dmrg_load_synthetic_part(ctx, nL, n, ntot, 0, left, right, seed, r, P)
            info = capi.dmrg_get_sigma_info(ctx)
            elems.append(info["op_elements"])
            y = np.zeros(size)
            capi.dmrg_sigma(ctx, -1, x, y)
            parts.append(y)
            with pytest.raises(capi.DMRGError):
                capi.dmrg_sigma_part(ctx, -1, 0, 2, x, np.zeros(size))
        finally:
            capi.dmrg_destroy(ctx)
    assert sum(elems) == total
    assert max(elems) <= 1.5 * total / P
    bL, bR, oL, oR, _ = synthetic_ops(left, right, nL, n, seed=seed)
    lay, _ = psi_layout(bL, bR, (ntot, 0))
    terms = nc_terms(nL, n)
    scale = np.abs(full).max()
    for r in range(P):
        ref = sigma_part(x, lay, terms, oL, oR, r, P)
        assert np.abs(parts[r] - ref).max() <= 1e-12 * scale, r
    assert np.abs(sum(parts) - full).max() <= 1e-12 * scale
