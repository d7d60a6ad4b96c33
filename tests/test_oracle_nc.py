"""Pins of the U(1) NC decomposition, sigma and the blocking formulas."""

import numpy as np
import pytest

from oracle.blocks import BlockOp
from oracle.fock import hamiltonian_fock
from oracle.nc import (Integrals, blocking_left, blocking_right, count_nc_terms,
                       fock_ops_exact, nc_terms)
from oracle.sigma import heff_dense, heff_diagonal, psi_layout, sigma_blocks
from synth import random_integrals


def _global_index(layout, bL, pL, bR, pR, nL):
    idx = []
    for qL, qR, mL, mR, off in layout:
        iL = bL.offsets[bL.index[qL]]
        iR = bR.offsets[bR.index[qR]]
        for a in range(mL):
            for b in range(mR):
                idx.append(pL[iL + a] | (pR[iR + b] << nL))
    return np.array(idx)


@pytest.mark.parametrize("K,nL,Q,seed", [(4, 4, (4, 0), 3), (4, 2, (3, 1), 1), (4, 6, (5, -1), 2),
                                         (3, 2, (2, 0), 8)])
def test_nc_sigma_equals_fock_hamiltonian(K, nL, Q, seed):
    t, v = random_integrals(K, seed)
    ints = Integrals(t, v)
    n = 2 * K
    bL, pL, oL = fock_ops_exact(ints, list(range(nL)), "L")
    bR, pR, oR = fock_ops_exact(ints, list(range(nL, n)), "R")
    H = hamiltonian_fock(t, v).toarray()
    lay, size = psi_layout(bL, bR, Q)
    idx = _global_index(lay, bL, pL, bR, pR, nL)
    x = np.random.default_rng(seed).standard_normal(size)
    terms = nc_terms(nL, n)
    assert len(terms) == count_nc_terms(nL, n - nL)
    s = sigma_blocks(x, lay, terms, oL, oR)
    ref = H[np.ix_(idx, idx)] @ x
    assert np.abs(s - ref).max() < 1e-12 * max(1.0, np.abs(ref).max())
    Hd = heff_dense(lay, terms, oL, oR)
    assert np.abs(Hd - Hd.T).max() < 1e-12
    assert np.abs(np.diag(Hd) - heff_diagonal(lay, terms, oL, oR)).max() < 1e-12


def test_term_count_formula():
    # 54|54 spatial orbitals = 108|108 spin orbitals: 2 + 432 + 11556 + 11664
    assert count_nc_terms(108, 108) == 23654
    assert len(nc_terms(108, 216)) == 23654


def _enlarged_index_left(E, chunks, bL, pL, nb):
    idx = np.zeros(E.total, dtype=np.int64)
    for Q in E.qs:
        base = E.offsets[E.index[Q]]
        for qb, ns, off in chunks[Q]:
            i0 = bL.offsets[bL.index[qb]]
            for a in range(bL.dim(qb)):
                idx[base + off + a] = pL[i0 + a] | (ns << nb)
    return idx


def _enlarged_index_right(E, chunks, bR, pR):
    idx = np.zeros(E.total, dtype=np.int64)
    for Q in E.qs:
        base = E.offsets[E.index[Q]]
        for qb, ns, off in chunks[Q]:
            i0 = bR.offsets[bR.index[qb]]
            for a in range(bR.dim(qb)):
                idx[base + off + a] = ns | (pR[i0 + a] << 2)
    return idx


def test_blocking_left_matches_fock_operators():
    K = 4
    t, v = random_integrals(K, 5)
    ints = Integrals(t, v)
    for site in range(1, K):
        bL, pL, oL = fock_ops_exact(ints, list(range(2 * site)), "L")
        bX, pX, oX = fock_ops_exact(ints, list(range(2 * site + 2)), "L")
        E, ch, enl = blocking_left(ints, bL, oL, site)
        pos = np.argsort(pX)[_enlarged_index_left(E, ch, bL, pL, 2 * site)]
        assert set(enl) == set(oX)
        for k, e in enl.items():
            D = e.assemble(E, ch).to_dense()
            assert np.abs(D - oX[k].to_dense()[np.ix_(pos, pos)]).max() < 1e-12, k


def test_blocking_right_matches_fock_operators():
    K = 4
    t, v = random_integrals(K, 6)
    ints = Integrals(t, v)
    n = 2 * K
    for site in range(0, K - 1):
        bR, pR, oR = fock_ops_exact(ints, list(range(2 * site + 2, n)), "R")
        bX, pX, oX = fock_ops_exact(ints, list(range(2 * site, n)), "R")
        E, ch, enl = blocking_right(ints, bR, oR, site)
        pos = np.argsort(pX)[_enlarged_index_right(E, ch, bR, pR)]
        assert set(enl) == set(oX)
        for k, e in enl.items():
            D = e.assemble(E, ch).to_dense()
            assert np.abs(D - oX[k].to_dense()[np.ix_(pos, pos)]).max() < 1e-12, k
