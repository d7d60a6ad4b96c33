"""The allocation-free sigma entry point (dmrg_sigma_noalloc).

It serves callers that cannot allocate device memory when they need a sigma
(a process whose HBM is reserved up front, or a loop that must not call
cudaMalloc/cudaFree). It runs the FP64 sigma kernel with its scratch in
fixed-size arrays compiled into the library. This file is collected last so
that a failure here stops a run only after every other test has run.
"""

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

TOL = 1e-12  # the FP64 sigma bar of the other GPU tests


def test_noalloc_sigma_equals_sigma_twice():
    """Two calls in a row (sharing, and reusing, the static scratch) give the
    oracle's sigma (plain per-term, per-block products on the CPU) within the
    FP64 bar, and the same result as dmrg_sigma."""
    import torch
    from oracle.nc import nc_terms
    from oracle.sigma import psi_layout, sigma_blocks, synthetic_ops
    from paper_2103_09976_gb300 import capi
    from synth import gaussian_sector_dims, mirrored_sectors, random_unit_vector
    left = gaussian_sector_dims(400, n_spatial=4, n_tot=8)
    right = mirrored_sectors(left, n_tot=8)
    ctx = capi.dmrg_create(device=0)
    try:
        capi.dmrg_load_synthetic(ctx, 8, 16, 8, 0, left, right, 5)
        n = capi.dmrg_psi_layout(ctx)["size"]
        x_h = random_unit_vector(n, 6)
        x = torch.from_numpy(x_h).cuda()
        ref = torch.zeros(n, dtype=torch.float64, device="cuda")
        capi.dmrg_sigma(ctx, -1, x, ref)
        capi.dmrg_sync(ctx)
        outs = []
        for _ in range(2):
            y = torch.full((n,), float("nan"), dtype=torch.float64, device="cuda")
            capi.dmrg_sigma_noalloc(ctx, -1, x, y)
            capi.dmrg_sync(ctx)
            outs.append(y.cpu().numpy())
    finally:
        capi.dmrg_destroy(ctx)
    bL, bR, oL, oR, _ = synthetic_ops(left, right, 8, 16, seed=5)
    lay, size = psi_layout(bL, bR, (8, 0))
    assert size == n
    want = sigma_blocks(x_h, lay, nc_terms(8, 16), oL, oR)
    scale = np.abs(want).max()
    r = ref.cpu().numpy()
    for y in outs:
        assert np.all(np.isfinite(y))
        assert np.abs(y - want).max() <= TOL * scale
        assert np.abs(y - r).max() <= TOL * scale


def test_noalloc_sweep_context_needs_resident_bond():
    """On a context built from integrals, a bond whose operators are not on
    the device is refused (building them would allocate); once dmrg_sigma
    has brought that bond in, the call gives dmrg_sigma's result."""
    import torch
    from paper_2103_09976_gb300 import capi
    from synth import random_integrals, random_unit_vector
    t, v = random_integrals(4, 7)
    ctx = capi.dmrg_create(device=0, seed=1)
    try:
        capi.dmrg_build_blocks(ctx, t, v, 4, 4, 0, 16)
        # right after dmrg_build_blocks the blocks of bond 0 exist; its
        # operators are built on the device by the first call that needs them
        n = capi.dmrg_psi_layout(ctx, 0)["size"]
        # bond 1 is not resident: refused before anything is read or built
        big = torch.zeros(1 << 16, dtype=torch.float64, device="cuda")
        with pytest.raises(capi.DMRGError) as e:
            capi.dmrg_sigma_noalloc(ctx, 1, big, torch.zeros_like(big))
        assert e.value.status == capi.DMRG_ESTATE
        x = torch.from_numpy(random_unit_vector(n, 3)).cuda()
        y = torch.zeros(n, dtype=torch.float64, device="cuda")
        ref = torch.zeros_like(y)
        capi.dmrg_sigma(ctx, 0, x, ref)
        capi.dmrg_sync(ctx)
        for _ in range(2):
            y.fill_(float("nan"))
            capi.dmrg_sigma_noalloc(ctx, 0, x, y)
            capi.dmrg_sync(ctx)
            r = ref.cpu().numpy()
            assert np.abs(y.cpu().numpy() - r).max() <= TOL * np.abs(r).max()
    finally:
        capi.dmrg_destroy(ctx)


def test_noalloc_rejects_host_pointers_and_oversized_problems():
    import torch
    from paper_2103_09976_gb300 import capi
    from synth import gaussian_sector_dims, mirrored_sectors
    ctx = capi.dmrg_create(device=0)
    try:
        left = gaussian_sector_dims(120, n_spatial=4, n_tot=8)
        capi.dmrg_load_synthetic(ctx, 8, 16, 8, 0, left, mirrored_sectors(left, n_tot=8), 1)
        n = capi.dmrg_psi_layout(ctx)["size"]
        with pytest.raises(capi.DMRGError) as e:
            capi.dmrg_sigma_noalloc(ctx, -1, np.zeros(n), np.zeros(n))
        assert e.value.status == capi.DMRG_EINVAL
        # 16 sectors, blocks up to ~125 wide: 5.3M doubles (42.5 MB) of partial tiles > 32 MiB
        left = gaussian_sector_dims(1400, n_spatial=3, n_tot=6)
        capi.dmrg_load_synthetic(ctx, 6, 12, 6, 0, left, mirrored_sectors(left, n_tot=6), 1)
        n = capi.dmrg_psi_layout(ctx)["size"]
        x = torch.zeros(n, dtype=torch.float64, device="cuda")
        y = torch.zeros(n, dtype=torch.float64, device="cuda")
        with pytest.raises(capi.DMRGError) as e:
            capi.dmrg_sigma_noalloc(ctx, -1, x, y)
        assert e.value.status == capi.DMRG_EINVAL and "32 MiB" in str(e.value)
    finally:
        capi.dmrg_destroy(ctx)
