"""CUDA-graph replay of sigma and the FP64 work-list autotuner.

Graph replay runs the same kernels on the same work list, so sigma and
Davidson results are bitwise those of direct launches. Autotuning changes
how tasks are grouped into items, so the tuned sigma is compared with the
oracle at the FP64 bar (1e-12 of max|sigma|) and must be deterministic."""

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

TOL = 1e-12


def _load(capi, M, nsp, ntot, seed, **opts):
    from synth import gaussian_sector_dims, mirrored_sectors
    left = gaussian_sector_dims(M, n_spatial=nsp, n_tot=ntot)
    right = mirrored_sectors(left, n_tot=ntot)
    ctx = capi.dmrg_create(device=0, **opts)
    capi.dmrg_load_synthetic(ctx, 2 * nsp, 4 * nsp, ntot, 0, left, right, seed)
    return ctx, left, right


@pytest.mark.parametrize("prec", ["FP64", "BF16X3"])
def test_graph_replay_is_bitwise_direct(prec):
    import torch
    from paper_2103_09976_gb300 import capi
    from synth import random_unit_vector
    outs = {}
    for graphs in (0, 1):
        ctx, _, _ = _load(capi, 400, 4, 8, 5, graphs=graphs, sigma_prec=getattr(capi, "DMRG_" + prec))
        try:
            n = capi.dmrg_psi_layout(ctx)["size"]
            x = torch.from_numpy(random_unit_vector(n, 7)).cuda()
            ys = []
            for _ in range(4):   # direct, capture, replay, replay
                y = torch.zeros(n, dtype=torch.float64, device="cuda")
                capi.dmrg_sigma(ctx, -1, x, y)
                capi.dmrg_sync(ctx)          # device pointers: the call is asynchronous on the library stream
                ys.append(y.cpu().numpy())
            yh = np.zeros(n)
            capi.dmrg_sigma(ctx, -1, x.cpu().numpy(), yh)   # host pointers: staged buffers
            e, it, conv = capi.dmrg_davidson(ctx, -1, None, 1e-10)
        finally:
            capi.dmrg_destroy(ctx)
        assert all(np.array_equal(ys[0], y) for y in ys[1:] + [yh])
        outs[graphs] = (ys[0], e, it)
    assert np.array_equal(outs[0][0], outs[1][0])
    assert outs[0][1] == outs[1][1] and outs[0][2] == outs[1][2]


def test_autotune_keeps_parity_and_determinism():
    from oracle.nc import nc_terms
    from oracle.sigma import psi_layout, sigma_blocks, synthetic_ops
    from paper_2103_09976_gb300 import capi
    from synth import random_unit_vector
    ctx, left, right = _load(capi, 1200, 3, 6, 3)
    try:
        w, c, ms = capi.dmrg_autotune(ctx)
        n = capi.dmrg_psi_layout(ctx)["size"]
        x = random_unit_vector(n, 13)
        y1, y2 = np.zeros(n), np.zeros(n)
        capi.dmrg_sigma(ctx, -1, x, y1)
        capi.dmrg_sigma(ctx, -1, x, y2)
    finally:
        capi.dmrg_destroy(ctx)
    assert w in (8, 16, 32) and c in (4096.0, 16384.0, 65536.0) and ms > 0
    assert np.array_equal(y1, y2)
    bL, bR, oL, oR, _ = synthetic_ops(left, right, 6, 12, seed=3)
    lay, _ = psi_layout(bL, bR, (6, 0))
    ref = sigma_blocks(x, lay, nc_terms(6, 12), oL, oR)
    assert np.abs(y1 - ref).max() <= TOL * np.abs(ref).max()


def test_tensor_core_autotune_keeps_parity_and_determinism():
    """At a mixed precision the tuner picks the tensor-core work split (items
    per SM and the fixed cost of a unit) and the producer setting, reported by
    dmrg_get_sigma_info; the tuned sigma stays within the
    BF16X3 bar of the oracle and bitwise repeatable, through direct launches
    and graph replays."""
    import torch
    from oracle.nc import nc_terms
    from oracle.sigma import psi_layout, sigma_blocks, synthetic_ops
    from paper_2103_09976_gb300 import capi
    from synth import random_unit_vector
    ctx, left, right = _load(capi, 1200, 3, 6, 3, sigma_prec=capi.DMRG_BF16X3)
    try:
        w, c, ms = capi.dmrg_autotune(ctx)
        info = capi.dmrg_get_sigma_info(ctx)
        n = capi.dmrg_psi_layout(ctx)["size"]
        x_h = random_unit_vector(n, 13)
        x = torch.from_numpy(x_h).cuda()
        ys = []
        for _ in range(3):   # direct, capture, replay
            y = torch.zeros(n, dtype=torch.float64, device="cuda")
            capi.dmrg_sigma(ctx, -1, x, y)
            capi.dmrg_sync(ctx)
            ys.append(y.cpu().numpy())
    finally:
        capi.dmrg_destroy(ctx)
    assert w in (4, 8, 16, 32) and c in (2.0 ** 20, 2.0 ** 22, 2.0 ** 24) and ms > 0
    assert (info["tc_items_per_sm"], info["tc_unit_cost"]) == (w, c) and info["tc_producers"] in (1, 3)
    assert all(np.array_equal(ys[0], y) for y in ys[1:])
    bL, bR, oL, oR, _ = synthetic_ops(left, right, 6, 12, seed=3)
    lay, _ = psi_layout(bL, bR, (6, 0))
    ref = sigma_blocks(x_h, lay, nc_terms(6, 12), oL, oR)
    assert np.abs(ys[0] - ref).max() <= 2e-6 * np.abs(ref).max()
