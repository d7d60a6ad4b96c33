"""Pins of the synthetic middle-bond sigma layout (random operator blocks)."""

import numpy as np

from oracle.blocks import Basis
from oracle.nc import Integrals, fock_ops_exact, nc_terms
from oracle.sigma import (heff_dense, heff_diagonal, psi_layout, sigma_blocks, sigma_flops,
                          synthetic_block_table, synthetic_op_specs, synthetic_ops,
                          synthetic_sigma_sampled)
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
    assert fl == _flops_by_shift_class(lay, nsp=54)


def _flops_by_shift_class(lay, nsp):
    """Independent count of the same work: terms grouped by the left shift
    (dN, d2Sz) they apply. With nsp spatial orbitals per side (2 nsp spin
    orbitals, half alpha), the NC terms per shift class are: B.Q with equal
    spins (0, 0): 2 (nsp^2); B.Q with opposite spins (0, +-2): nsp^2 each;
    a+.R^R and (R^L)^T.a (+-1, +-1): 2 nsp each (and the same for their
    conjugates); A.P with opposite spins (+-2, 0): nsp^2 each; A.P with equal
    spins (+-2, +-2): nsp (nsp - 1) / 2 each. H_L x 1 and 1 x H_R cost
    2 m^2 n and 2 m n^2 per block."""
    blk = {qL: (m, n) for qL, qR, m, n, off in lay}
    count = {(0, 0): 2 * nsp * nsp, (0, 2): nsp * nsp, (0, -2): nsp * nsp,
             (2, 0): nsp * nsp, (-2, 0): nsp * nsp}
    for dn in (1, -1):
        for ds in (1, -1):
            count[(dn, ds)] = 2 * nsp
    for dn in (2, -2):
        for ds in (2, -2):
            count[(dn, ds)] = nsp * (nsp - 1) // 2
    total = sum(2 * m * m * n + 2 * m * n * n for m, n in blk.values())
    for qo, (mo, no) in blk.items():
        for (dn, ds), T in count.items():
            qi = (qo[0] - dn, qo[1] - ds)
            if qi not in blk:
                continue
            m, n = blk[qi]
            total += T * min(2 * mo * m * n + 2 * mo * n * no, 2 * m * n * no + 2 * mo * m * no)
    return total


def test_sigma_flops_hand_count():
    """sigma_flops on a layout small enough to count by hand. Left sectors
    (0,0) dim 2 and (1,1) dim 3; right (1,1) dim 4 and (0,0) dim 5; target
    (1,1), so psi has blocks 2x4 (q_L = (0,0)) and 3x5 (q_L = (1,1)).
    Terms and their costs:
      H_L x 1:  2*2*2*4 + 2*3*3*5                      = 32 + 90  = 122
      1 x H_R:  2*2*4*4 + 2*3*5*5                      = 64 + 150 = 214
      a+ x R (shifts (1,1), (-1,-1)), block 2x4 -> 3x5:
          min(2*3*2*4 + 2*3*4*5, 2*2*4*5 + 2*3*2*5)  = min(168, 140) = 140
      its conjugate (transposes), block 3x5 -> 2x4:
          min(2*2*3*5 + 2*2*5*4, 2*3*5*4 + 2*2*3*4)  = min(140, 168) = 140
    Total 616. The two conjugates take the cheaper order from opposite
    sides, so picking max instead of min, or swapping m and n, changes it."""
    bL = Basis([((0, 0), 2), ((1, 1), 3)])
    bR = Basis([((0, 0), 5), ((1, 1), 4)])
    lay, size = psi_layout(bL, bR, (1, 1))
    assert [(m, n) for _, _, m, n, _ in lay] == [(2, 4), (3, 5)] and size == 23
    dqL = {"H": (0, 0), "c": (1, 1)}
    dqR = {"H": (0, 0), "r": (-1, -1)}
    terms = [("H", False, None, False, 1.0), (None, False, "H", False, 1.0),
             ("c", False, "r", False, 1.0), ("c", True, "r", True, -1.0)]
    assert sigma_flops(lay, terms, dqL, dqR, bL, bR) == 616
    assert sigma_flops(lay, terms[:2], dqL, dqR, bL, bR) == 122 + 214


def test_flops_by_shift_class_matches_term_loop_small():
    """The shift-class count above and the oracle's per-term loop agree on
    small middle-bond layouts (and so the class counts are those of nc_terms)."""
    for nsp, ntot, M in ((3, 6, 24), (4, 8, 40), (5, 10, 70)):
        left = gaussian_sector_dims(M, n_spatial=nsp, n_tot=ntot)
        right = mirrored_sectors(left, n_tot=ntot)
        bL = Basis([((a, b), d) for a, b, d in left])
        bR = Basis([((a, b), d) for a, b, d in right])
        lay, _ = psi_layout(bL, bR, (ntot, 0))
        specs = synthetic_op_specs(2 * nsp, 4 * nsp)
        dqL = {k: dq for s, k, dq, _ in specs if s == "L"}
        dqR = {k: dq for s, k, dq, _ in specs if s == "R"}
        fl = sigma_flops(lay, nc_terms(2 * nsp, 4 * nsp), dqL, dqR, bL, bR)
        assert fl == _flops_by_shift_class(lay, nsp)


def test_sampled_sigma_equals_full_sigma():
    """synthetic_sigma_sampled (rows of operator blocks drawn one by one from
    their counters, transposed uses read as columns, symmetric operators from
    their upper triangle) equals sigma_blocks on the full synthetic operators,
    entry by entry, for several small middle-bond problems and seeds. Every
    output block is sampled; transposed conjugate terms, the symmetric H, B_pp
    and Q_pp, and blocks that some terms do not reach all occur."""
    cases = [(3, 6, 0, 24, 1), (3, 6, 0, 30, 7), (4, 8, 0, 40, 2), (4, 7, 1, 36, 5)]
    for nsp, ntot, tsz, M, seed in cases:
        left = gaussian_sector_dims(M, n_spatial=nsp, n_tot=ntot, two_sz_tot=tsz)
        right = mirrored_sectors(left, n_tot=ntot, two_sz_tot=tsz)
        nL, n = 2 * nsp, 4 * nsp
        bL, bR, oL, oR, _ = synthetic_ops(left, right, nL, n, seed)
        lay, size = psi_layout(bL, bR, (ntot, tsz))
        x = np.random.default_rng(seed + 100).standard_normal(size)
        full = sigma_blocks(x, lay, nc_terms(nL, n), oL, oR)
        rng = np.random.default_rng(seed)
        samples = []
        for qL, qR, m, nn, off in lay:
            rows = np.sort(rng.choice(m, size=max(1, (m + 1) // 2), replace=False))
            cols = np.sort(rng.choice(nn, size=max(1, (nn + 1) // 2), replace=False))
            samples.append((qL, rows, cols))
        got = synthetic_sigma_sampled(left, right, nL, n, seed, (ntot, tsz), x, samples)
        scale = np.abs(full).max()
        assert scale > 1.0
        for qL, rows, cols in samples:
            _, _, m, nn, off = next(b for b in lay if b[0] == qL)
            ref = full[off:off + m * nn].reshape(m, nn)[np.ix_(rows, cols)]
            assert np.abs(got[qL] - ref).max() <= 1e-13 * scale, (nsp, M, seed, qL)
