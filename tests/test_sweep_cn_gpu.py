"""GPU sweeps with the mixed NC/CN partition (Sec. III.A, App. B Eq. h-cn)
against the oracle: full bond dimension reproduces FCI at every cut;
CN-form blocks and the blocks made by the normal-to-complementary
transformation at the cut equal the oracle's, initial and swept."""

import json
import os

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

GOLD = os.path.join(os.path.dirname(__file__), "golden", "fci_energies.json")


def form_keys(nL, n, left, cn):
    """Oracle operator keys in the library's canonical order for a block of
    either form (pairs over [0, nL) in NC form, over [nL, n) in CN form)."""
    keys = ["H"]
    if left:
        keys += [("cd", p) for p in range(nL)] + [("RL", p) for p in range(nL, n)]
    else:
        keys += [("d", p) for p in range(nL, n)] + [("RR", p) for p in range(nL)]
    lo, hi = (nL, n) if cn else (0, nL)
    normal = left != cn
    keys += [("A" if normal else "P", p, r) for p in range(lo, hi) for r in range(p + 1, hi)]
    keys += [("B" if normal else "Q", p, q) for p in range(lo, hi) for q in range(p, hi)]
    return keys


def _compare_block(capi, ctx, side, j, basis, ops, K, cut, tol):
    q, d, nops = capi.dmrg_block_info(ctx, side, j)
    assert [tuple(x) for x in q.tolist()] == list(basis.qs), (side, j)
    assert d.tolist() == list(basis.dims), (side, j)
    keys = form_keys(2 * j, 2 * K, side == 0, j > cut)
    assert nops == len(keys) and set(keys) == set(ops), (side, j)
    for k, key in enumerate(keys):
        got = capi.dmrg_block_read(ctx, side, j, k)
        ref = ops[key].to_dense()
        assert np.abs(got - ref).max() <= tol * max(1.0, np.abs(ref).max()), (side, j, key)


@pytest.mark.parametrize("K,N,s,cut", [(5, 5, 1, 2), (5, 4, 0, 0), (4, 3, -1, 1), (5, 6, 0, 3)])
def test_mixed_full_m_sweeps_equal_fci(K, N, s, cut):
    from oracle.fock import fci_energy
    from paper_2103_09976_gb300 import capi
    from synth import random_integrals
    t, v = random_integrals(K, 9)
    ref = fci_energy(t, v, N, s)
    M = 4 ** K
    ctx = capi.dmrg_create(device=0, dav_max_iter=400, seed=1, mixed_cut=cut)
    try:
        capi.dmrg_build_blocks(ctx, t, v, K, N, s, M)
        e, d = capi.dmrg_sweep(ctx, [M] * 3, 1e-12)
        log = capi.dmrg_sweep_log(ctx)
    finally:
        capi.dmrg_destroy(ctx)
    assert np.all(np.abs(e - ref) < 1e-9), (e, ref)
    assert all(g["energy"] - ref < 1e-9 for g in log)


def test_mixed_config1_sweeps_equal_stored_fci():
    """K=8, N=8, 2Sz=0, seed 0, M=256, 4 sweeps, tol 1e-10, NC for steps whose
    enlarged left block holds at most K/2 = 4 orbitals and CN beyond."""
    from paper_2103_09976_gb300 import capi
    from synth import random_integrals
    gold = json.load(open(GOLD))["cfg1"]
    t, v = random_integrals(8, 0)
    ctx = capi.dmrg_create(device=0, dav_max_iter=400, seed=0, mixed_cut=4)
    try:
        capi.dmrg_build_blocks(ctx, t, v, 8, 8, 0, 256)
        e, d = capi.dmrg_sweep(ctx, [256] * 4, 1e-10)
    finally:
        capi.dmrg_destroy(ctx)
    assert np.all(np.abs(e - gold["energy"]) < 1e-9), (e, gold["energy"])


def test_mixed_initial_blocks_equal_oracle():
    """Initial right blocks at M_init=8 with cut 2: CN-form blocks right of
    the cut, the transformed block R[2] and NC-form blocks left of it equal
    the oracle's operator by operator."""
    from oracle.dmrg import PlainDMRG
    from paper_2103_09976_gb300 import capi
    from synth import random_integrals
    K, cut = 5, 2
    t, v = random_integrals(K, 7)
    ora = PlainDMRG(t, v, 4, 2, seed=1, cut=cut)
    ora.build_blocks(8)
    ctx = capi.dmrg_create(device=0, seed=1, mixed_cut=cut)
    try:
        capi.dmrg_build_blocks(ctx, t, v, K, 4, 2, 8)
        for j in range(1, K + 1):
            _compare_block(capi, ctx, 1, j, ora.R[j][0], ora.R[j][1], K, cut, 1e-12)
    finally:
        capi.dmrg_destroy(ctx)


@pytest.mark.parametrize("cut", [2, 3])
def test_mixed_truncated_sweeps_follow_oracle(cut):
    """M=8 sweeps with the mixed partition: per-step energies and discarded
    weights, and every left and right block after the sweeps, follow the
    oracle's mixed NC/CN DMRG (Davidson to a squared residual of 1e-20)."""
    from oracle.dmrg import PlainDMRG
    from paper_2103_09976_gb300 import capi
    from synth import random_integrals
    K = 5
    t, v = random_integrals(K, 7)
    ora = PlainDMRG(t, v, 4, 2, seed=1, dav_tol=1e-20, dav_max_iter=400, cut=cut)
    ora.build_blocks(8)
    e_ref, d_ref = ora.sweep([8, 8, 8])
    ctx = capi.dmrg_create(device=0, dav_max_iter=400, seed=1, mixed_cut=cut)
    try:
        capi.dmrg_build_blocks(ctx, t, v, K, 4, 2, 8)
        e, d = capi.dmrg_sweep(ctx, [8, 8, 8], 1e-20)
        log = capi.dmrg_sweep_log(ctx)
        for i in range(1, K):
            _compare_block(capi, ctx, 0, i, ora.L[i][0], ora.L[i][1], K, cut, 1e-7)
        for j in range(1, K):
            _compare_block(capi, ctx, 1, j, ora.R[j][0], ora.R[j][1], K, cut, 1e-7)
    finally:
        capi.dmrg_destroy(ctx)
    assert len(log) == len(ora.log) == 3 * (K - 1)
    for g, o in zip(log, ora.log):
        assert (g["site"], g["forward"], g["psi_size"]) == (o["i"], int(o["forward"]), o["dim"])
        assert abs(g["energy"] - o["energy"]) < 1e-9, (g, o)
        assert abs(g["discarded"] - o["discarded"]) <= 1e-6 * o["discarded"] + 1e-14, (g, o)
    assert np.all(np.abs(e - np.array(e_ref)) < 1e-9), (e, e_ref)


def test_mixed_and_nc_give_the_same_step_energies():
    """The partition changes how H_eff is assembled, not H_eff: a K=8 run at
    M=24 gives the same first-sweep step energies with NC everywhere and
    with the mixed partition (cut 4), on the GPU."""
    from paper_2103_09976_gb300 import capi
    from synth import random_integrals
    K = 8
    t, v = random_integrals(K, 3)
    runs = []
    for cut in (-1, 4):
        ctx = capi.dmrg_create(device=0, dav_max_iter=400, seed=2, mixed_cut=cut)
        try:
            capi.dmrg_build_blocks(ctx, t, v, K, 8, 0, 24)
            capi.dmrg_sweep(ctx, [24], 1e-16)
            runs.append([g["energy"] for g in capi.dmrg_sweep_log(ctx)])
        finally:
            capi.dmrg_destroy(ctx)
    assert np.abs(np.array(runs[0]) - np.array(runs[1])).max() < 1e-8


def test_cn_bond_sigma_and_parts_match_oracle():
    """At a CN bond (cut 0: every step is CN; bond 0's enlarged left block
    comes from the normal-to-complementary transformation of the vacuum and
    the right block is in CN form): the GPU sigma and its sub-Hamiltonian
    parts (Eq. proc-def-cn) equal the oracle's on the same psi."""
    from oracle.cn import cn_terms
    from oracle.dmrg import PlainDMRG
    from oracle.sigma import psi_layout, sigma_blocks, sigma_part
    from paper_2103_09976_gb300 import capi
    from synth import random_integrals, random_unit_vector
    K, N, s, M, P = 5, 5, 1, 10, 3
    t, v = random_integrals(K, 5)
    ora = PlainDMRG(t, v, N, s, seed=4, cut=0)
    ora.build_blocks(M)
    EL, oL, ER, oR = ora.enlarged(0)
    lay, size = psi_layout(EL, ER, (N, s))
    terms = cn_terms(2, 2 * K)
    x = random_unit_vector(size, 7)
    ref = sigma_blocks(x, lay, terms, oL, oR)
    ctx = capi.dmrg_create(device=0, seed=4, mixed_cut=0)
    try:
        capi.dmrg_build_blocks(ctx, t, v, K, N, s, M)
        assert capi.dmrg_psi_layout(ctx, 0)["size"] == size
        y = np.zeros(size)
        capi.dmrg_sigma(ctx, 0, x, y)
        parts = []
        for r in range(P):
            z = np.zeros(size)
            capi.dmrg_sigma_part(ctx, 0, r, P, x, z)
            parts.append(z)
    finally:
        capi.dmrg_destroy(ctx)
    scale = np.abs(ref).max()
    assert np.abs(y - ref).max() <= 1e-12 * scale
    for r in range(P):
        assert np.abs(parts[r] - sigma_part(x, lay, terms, oL, oR, r, P)).max() <= 1e-12 * scale, r
    assert np.abs(sum(parts) - y).max() <= 1e-12 * scale
