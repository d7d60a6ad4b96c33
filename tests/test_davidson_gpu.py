"""GPU Davidson (FP64 control path) against the exact lowest eigenvalue of the
explicit H_eff (oracle), for the FP64 sigma and the tensor-core sigma.

FP64: the converged Ritz value of a symmetric matrix with squared residual
norm rr < tol is within rr / gap of an eigenvalue; with tol = 1e-20 and gaps
~1e-2 this is ~1e-18 - the bar 1e-9 is the target accuracy for energies.
BF16X3: the sigma carries a relative error ~1e-6 (see test_sigma_tc_gpu), so
the Ritz value is that of a perturbed matrix: |dE| <~ ||dH|| ~ 1e-6 |E|.
"""

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _exact(left, right, nL, n, Q, seed):
    from oracle.nc import nc_terms
    from oracle.sigma import heff_dense, psi_layout, synthetic_ops
    bL, bR, oL, oR, _ = synthetic_ops(left, right, nL, n, seed=seed)
    lay, size = psi_layout(bL, bR, Q)
    H = heff_dense(lay, nc_terms(nL, n), oL, oR)
    w, V = np.linalg.eigh(H)
    return w, V


@pytest.mark.parametrize("prec,bar", [(0, 1e-9), (2, 1e-5), (3, 1e-5)])
def test_davidson_lowest_eigenvalue(prec, bar):
    from paper_2103_09976_gb300 import capi
    from synth import gaussian_sector_dims, mirrored_sectors, random_unit_vector
    left = gaussian_sector_dims(60, n_spatial=4, n_tot=8)
    right = mirrored_sectors(left, n_tot=8)
    w, V = _exact(left, right, 8, 16, (8, 0), 3)
    ctx = capi.dmrg_create(device=0, sigma_prec=prec, dav_max_iter=600, dav_max_space=24)
    try:
        capi.dmrg_load_synthetic(ctx, 8, 16, 8, 0, left, right, 3)
        n = capi.dmrg_psi_layout(ctx)["size"]
        x = np.zeros(n)
        e, it, conv = capi.dmrg_davidson(ctx, -1, random_unit_vector(n, 9), 1e-20 if prec == 0 else 1e-9, x)
        e2, it2, conv2 = capi.dmrg_davidson(ctx, -1, None, 1e-20 if prec == 0 else 1e-9)
    finally:
        capi.dmrg_destroy(ctx)
    assert conv and conv2
    assert abs(e - w[0]) <= bar * max(1.0, abs(w[0])), (e, w[0])
    assert abs(e2 - w[0]) <= bar * max(1.0, abs(w[0]))
    # eigenvector: unit norm, overlap with the exact ground state
    assert abs(np.linalg.norm(x) - 1.0) < 1e-10
    if w[1] - w[0] > 1e-6:
        assert abs(V[:, 0] @ x) > 1.0 - (1e-8 if prec == 0 else 1e-3)


def test_davidson_iteration_limit_reports_enoconv():
    """dav_max_iter reached: DMRG_ENOCONV, with the best Ritz pair still
    returned; a Ritz value of a symmetric matrix is an upper bound of its
    lowest eigenvalue."""
    from paper_2103_09976_gb300 import capi
    from synth import gaussian_sector_dims, mirrored_sectors
    left = gaussian_sector_dims(60, n_spatial=4, n_tot=8)
    right = mirrored_sectors(left, n_tot=8)
    w, _ = _exact(left, right, 8, 16, (8, 0), 3)
    ctx = capi.dmrg_create(device=0, dav_max_iter=3)
    try:
        capi.dmrg_load_synthetic(ctx, 8, 16, 8, 0, left, right, 3)
        n = capi.dmrg_psi_layout(ctx)["size"]
        x = np.zeros(n)
        e, it, conv = capi.dmrg_davidson(ctx, -1, None, 1e-20, x)
    finally:
        capi.dmrg_destroy(ctx)
    assert not conv and it == 3
    assert np.isfinite(e) and e >= w[0] - 1e-9 * abs(w[0])
    assert abs(np.linalg.norm(x) - 1.0) < 1e-10
