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
    import torch
    from paper_2103_09976_gb300 import capi
    from synth import gaussian_sector_dims, mirrored_sectors, random_unit_vector
    left = gaussian_sector_dims(400, n_spatial=4, n_tot=8)
    right = mirrored_sectors(left, n_tot=8)
    ctx = capi.dmrg_create(device=0)
    try:
        capi.dmrg_load_synthetic(ctx, 8, 16, 8, 0, left, right, 5)
        n = capi.dmrg_psi_layout(ctx)["size"]
        x = torch.from_numpy(random_unit_vector(n, 6)).cuda()
        ref = torch.zeros(n, dtype=torch.float64, device="cuda")
        capi.dmrg_sigma(ctx, -1, x, ref)
        capi.dmrg_sync(ctx)
        outs = []
        for _ in range(2):  # two calls in a row share (and reuse) the static scratch
            y = torch.full((n,), float("nan"), dtype=torch.float64, device="cuda")
            capi.dmrg_sigma_noalloc(ctx, -1, x, y)
            capi.dmrg_sync(ctx)
            outs.append(y.cpu().numpy())
    finally:
        capi.dmrg_destroy(ctx)
    r = ref.cpu().numpy()
    scale = np.abs(r).max()
    for y in outs:
        assert np.all(np.isfinite(y))
        assert np.abs(y - r).max() <= TOL * scale


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
