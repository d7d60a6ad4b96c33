"""GPU two-site sweeps (blocking, Davidson, decimation, transformation)
against the oracle: full bond dimension reproduces FCI (to 1e-9, the FP64
energy target), truncated sweeps follow the oracle's plain DMRG (same seeds,
same counter-based guesses), sector tables are bit-exact."""

import json
import os

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

GOLD = os.path.join(os.path.dirname(__file__), "golden", "fci_energies.json")


def _ctx(capi, **kw):
    return capi.dmrg_create(device=0, dav_max_iter=400, **kw)


def nc_keys(nL, n, left):
    """Oracle operator keys in the library's canonical NC order."""
    keys = ["H"]
    if left:
        keys += [("cd", p) for p in range(nL)] + [("RL", p) for p in range(nL, n)]
    else:
        keys += [("d", p) for p in range(nL, n)] + [("RR", p) for p in range(nL)]
    keys += [("A" if left else "P", p, r) for p in range(nL) for r in range(p + 1, nL)]
    keys += [("B" if left else "Q", p, q) for p in range(nL) for q in range(p, nL)]
    return keys


def _compare_block(capi, ctx, side, j, basis, ops, K, tol, gauge_free):
    q, d, nops = capi.dmrg_block_info(ctx, side, j)
    assert [tuple(x) for x in q.tolist()] == list(basis.qs), (side, j)
    assert d.tolist() == list(basis.dims), (side, j)
    keys = nc_keys(2 * j, 2 * K, side == 0)
    assert nops == len(keys) and set(keys) == set(ops)
    for k, key in enumerate(keys):
        got = capi.dmrg_block_read(ctx, side, j, k)
        ref = ops[key].to_dense()
        if gauge_free:  # kept singular vectors carry a free sign each
            got, ref = np.abs(got), np.abs(ref)
        assert np.abs(got - ref).max() <= tol * max(1.0, np.abs(ref).max()), (side, j, key)


@pytest.mark.parametrize("K,N,s,M", [(4, 4, 0, 16), (5, 5, 1, 32)])
def test_full_m_sweeps_equal_fci(K, N, s, M):
    from oracle.fock import fci_energy
    from paper_2103_09976_gb300 import capi
    from synth import random_integrals
    t, v = random_integrals(K, 7)
    ref = fci_energy(t, v, N, s)
    ctx = _ctx(capi, seed=1)
    try:
        capi.dmrg_build_blocks(ctx, t, v, K, N, s, M)
        e, d = capi.dmrg_sweep(ctx, [M] * 3, 1e-12)
        log = capi.dmrg_sweep_log(ctx)
    finally:
        capi.dmrg_destroy(ctx)
    assert np.all(np.abs(e - ref) < 1e-9), (e, ref)
    assert np.all(d < 1e-20)
    # at full M the previous ground state carried to the next bond is exact,
    # so every solve after the first sweep starts converged
    assert all(g["iters"] <= 3 for g in log[K - 1:]), [g["iters"] for g in log]


def test_initial_blocks_equal_oracle():
    """Truncated initial right blocks (M_init=8 < full): same sectors, and the
    same operator matrices (the random bases are fixed by the counter-based
    generator and the Gram-Schmidt orientation)."""
    from oracle.dmrg import PlainDMRG
    from paper_2103_09976_gb300 import capi
    from synth import random_integrals
    K = 5
    t, v = random_integrals(K, 7)
    ora = PlainDMRG(t, v, 4, 2, seed=1)
    ora.build_blocks(8)
    ctx = _ctx(capi, seed=1)
    try:
        capi.dmrg_build_blocks(ctx, t, v, K, 4, 2, 8)
        for j in range(1, K + 1):
            _compare_block(capi, ctx, 1, j, ora.R[j][0], ora.R[j][1], K, 1e-12, False)
    finally:
        capi.dmrg_destroy(ctx)


def test_truncated_sweeps_follow_oracle():
    """M=8 sweeps: per-step energies, kept counts and discarded weights follow
    the oracle's plain DMRG. Each Davidson stops at a squared residual below
    1e-20, so the two eigenvectors agree to about 1e-10 and the truncated
    bases to the same order; energies then agree far inside 1e-9."""
    from oracle.dmrg import PlainDMRG
    from paper_2103_09976_gb300 import capi
    from synth import random_integrals
    K = 5
    t, v = random_integrals(K, 7)
    ora = PlainDMRG(t, v, 4, 2, seed=1, dav_tol=1e-20, dav_max_iter=400)
    ora.build_blocks(8)
    e_ref, d_ref = ora.sweep([8, 8, 8, 8])
    ctx = _ctx(capi, seed=1)
    try:
        capi.dmrg_build_blocks(ctx, t, v, K, 4, 2, 8)
        e, d = capi.dmrg_sweep(ctx, [8, 8, 8, 8], 1e-20)
        log = capi.dmrg_sweep_log(ctx)
        for i in range(1, K):
            _compare_block(capi, ctx, 0, i, ora.L[i][0], ora.L[i][1], K, 1e-7, False)
        for j in range(1, K):
            _compare_block(capi, ctx, 1, j, ora.R[j][0], ora.R[j][1], K, 1e-7, False)
    finally:
        capi.dmrg_destroy(ctx)
    assert len(log) == len(ora.log) == 4 * (K - 1)
    for g, o in zip(log, ora.log):
        assert (g["site"], g["forward"], g["psi_size"]) == (o["i"], int(o["forward"]), o["dim"])
        assert g["converged"] and o["converged"]
        assert abs(g["iters"] - o["nmv"]) <= 2, (g, o)   # same carried guess on both sides
        assert abs(g["energy"] - o["energy"]) < 1e-9, (g, o)
        assert abs(g["discarded"] - o["discarded"]) <= 1e-6 * o["discarded"] + 1e-14, (g, o)
    assert np.all(np.abs(e - np.array(e_ref)) < 1e-9), (e, e_ref)


def test_bond_layouts_and_energies_match_oracle():
    """After the initial blocks: psi layout at every bond is bit-exact, and the
    lowest eigenvalue of H_eff at every bond agrees (gauge-invariant)."""
    from oracle.dmrg import PlainDMRG
    from oracle.sigma import psi_layout
    from paper_2103_09976_gb300 import capi
    from synth import random_integrals
    K, N, s, M = 5, 5, 1, 12
    t, v = random_integrals(K, 4)
    ora = PlainDMRG(t, v, N, s, seed=3, dav_tol=1e-13)
    ora.build_blocks(M)
    ctx = _ctx(capi, seed=3)
    try:
        capi.dmrg_build_blocks(ctx, t, v, K, N, s, M)
        # bond 0 uses L_0 (vacuum) and R_2 from the initial blocks
        EL, oL, ER, oR = ora.enlarged(0)
        lay, size = psi_layout(EL, ER, (N, s))
        g = capi.dmrg_psi_layout(ctx, 0)
        assert g["size"] == size and len(g["m_l"]) == len(lay)
        for k, (qL, qR, mL, mR, off) in enumerate(lay):
            assert tuple(g["q_l"][k]) == qL and g["m_l"][k] == mL and g["m_r"][k] == mR and g["offset"][k] == off
        th, x, layout, nmv, conv = ora.solve(0, 0, EL, oL, ER, oR)
        e, it, conv2 = capi.dmrg_davidson(ctx, 0, None, 1e-14)
    finally:
        capi.dmrg_destroy(ctx)
    assert conv2 and abs(e - th) < 1e-9


def test_config1_sweeps_equal_stored_fci():
    """K=8, N=8, 2Sz=0, seed 0, M=256 (full at every bond), 4 sweeps, tol 1e-10."""
    from paper_2103_09976_gb300 import capi
    from synth import random_integrals
    gold = json.load(open(GOLD))["cfg1"]
    t, v = random_integrals(8, 0)
    ctx = _ctx(capi, seed=0)
    try:
        capi.dmrg_build_blocks(ctx, t, v, 8, 8, 0, 256)
        e, d = capi.dmrg_sweep(ctx, [256] * 4, 1e-10)
    finally:
        capi.dmrg_destroy(ctx)
    assert np.all(np.abs(e - gold["energy"]) < 1e-9), (e, gold["energy"])


def test_noise_and_keep_one_per_q_follow_oracle():
    """Perturbative noise (seeded, same stream on both sides) and one kept
    state per quantum number: step-by-step energies, kept counts and
    discarded weights equal the oracle's."""
    from oracle.dmrg import PlainDMRG
    from paper_2103_09976_gb300 import capi
    from synth import random_integrals
    K = 5
    t, v = random_integrals(K, 7)
    ora = PlainDMRG(t, v, 4, 2, seed=1, dav_tol=1e-20, dav_max_iter=400, noise=1e-2, keep_one_per_q=True)
    ora.build_blocks(3)
    ora.sweep([3, 3, 3])
    assert max(l["kept"] for l in ora.log) > 3          # extra states per quantum number were kept
    ctx = _ctx(capi, seed=1, noise=1e-2, keep_one_per_q=1)
    try:
        capi.dmrg_build_blocks(ctx, t, v, K, 4, 2, 3)
        capi.dmrg_sweep(ctx, [3, 3, 3], 1e-20)
        log = capi.dmrg_sweep_log(ctx)
    finally:
        capi.dmrg_destroy(ctx)
    assert len(log) == len(ora.log)
    for g, o in zip(log, ora.log):
        assert (g["site"], g["psi_size"], g["kept"]) == (o["i"], o["dim"], o["kept"])
        assert abs(g["energy"] - o["energy"]) < 1e-9, (g, o)
        assert abs(g["discarded"] - o["discarded"]) <= 1e-6 * o["discarded"] + 1e-14, (g, o)
