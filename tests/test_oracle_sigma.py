"""Pins of the synthetic middle-bond sigma layout (random operator blocks)."""

import numpy as np

from oracle.blocks import Basis
from oracle.nc import Integrals, fock_ops_exact, nc_terms
from oracle.sigma import (heff_dense, heff_diagonal, psi_layout, sigma_blocks, sigma_flops,
                          synthetic_block_table, synthetic_op_specs, synthetic_ops)
from synth import gaussian_sector_dims, mirrored_sectors, random_integrals


def _small_layout(M=24, nsp=3, ntot=6):
    left = gaussian_sector_dims(M, n_spatial=nsp, n_tot=ntot)
    right = mirrored_sectors(left, n_tot=ntot)
    return left, right, 2 * nsp, 4 * nsp


def test_spec_shifts_equal_physical_operator_shifts():
    # the stored-operator table must carry the shifts of the physical
    # operators of the same name (exact Fock-space matrices)
    t, v = random_integrals(3, 1)
    ints = Integrals(t, v)
    _, _, oL = fock_ops_exact(ints, [0, 1, 2, 3], "L")
    _, _, oR = fock_ops_exact(ints, [4, 5], "R")
    for side, key, dq, sym in synthetic_op_specs(4, 6):
        ops = oL if side == "L" else oR
        assert ops[key].dq == dq, (side, key)
        if sym:
            D = ops[key].to_dense()
            assert np.abs(D - D.T).max() < 1e-14


def test_synthetic_heff_is_symmetric_and_consistent():
    left, right, nL, n = _small_layout()
    bL, bR, oL, oR, total = synthetic_ops(left, right, nL, n, seed=1)
    Qtot = (6, 0)
    lay, size = psi_layout(bL, bR, Qtot)
    terms = nc_terms(nL, n)
    H = heff_dense(lay, terms, oL, oR)
    assert np.abs(H).max() > 1.0
    assert np.abs(H - H.T).max() < 1e-12 * np.abs(H).max()
    assert np.abs(np.diag(H) - heff_diagonal(lay, terms, oL, oR)).max() < 1e-12
    x = np.random.default_rng(3).standard_normal(size)
    assert np.abs(H @ x - sigma_blocks(x, lay, terms, oL, oR)).max() < 1e-11


def test_synthetic_values_follow_counter_layout():
    left, right, nL, n = _small_layout()
    bL, bR, oL, oR, total = synthetic_ops(left, right, nL, n, seed=1)
    specs = synthetic_op_specs(nL, n)
    table, total2 = synthetic_block_table(specs, bL, bR)
    assert total == total2
    # every stored element is drawn once: the flat layout tiles [0, total)
    spans = sorted((off, r * c) for blks in table for (_, _, r, c, off) in blks)
    pos = 0
    for off, ln in spans:
        assert off == pos
        pos += ln
    assert pos == total
    # partial builds reuse the canonical counters
    _, _, oL2, oR2, _ = synthetic_ops(left, right, nL, n, seed=1, only={("R", ("P", 0, 2))})
    for q, b in oR2[("P", 0, 2)].blocks.items():
        assert np.array_equal(b, oR[("P", 0, 2)].blocks[q])


def test_middle_bond_workload_sizes():
    """Sizes of the K=108, N=30 middle-bond workload at M=2000 (sector rule of
    synth.gaussian_sector_dims): 104 sectors, |psi| = 106004, 23654 terms."""
    left = gaussian_sector_dims(2000)
    right = mirrored_sectors(left)
    bL = Basis([((a, b), d) for a, b, d in left])
    bR = Basis([((a, b), d) for a, b, d in right])
    lay, size = psi_layout(bL, bR, (30, 0))
    assert len(lay) == 104 and size == 106004
    specs = synthetic_op_specs(108, 216)
    dqL = {k: dq for s, k, dq, _ in specs if s == "L"}
    dqR = {k: dq for s, k, dq, _ in specs if s == "R"}
    terms = nc_terms(108, 216)
    assert len(terms) == 23654
    fl = sigma_flops(lay, terms, dqL, dqR, bL, bR)
    assert 0.56e12 < fl < 0.58e12
