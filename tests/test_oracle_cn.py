"""Pins of the U(1) CN decomposition, the CN blocking formulas, the
normal-to-complementary transformation and mixed NC/CN sweeps (oracle)."""

import numpy as np
import pytest

from oracle.cn import (blocking_left_cn, blocking_right_cn, cn_terms, count_cn_terms,
                       vacuum_right_cn)
from oracle.dmrg import PlainDMRG
from oracle.fock import fci_energy, hamiltonian_fock
from oracle.nc import Integrals, fock_ops_exact, nc_terms
from oracle.sigma import heff_dense, heff_diagonal, psi_layout, sigma_blocks
from synth import random_integrals

from test_oracle_nc import _enlarged_index_left, _enlarged_index_right, _global_index


@pytest.mark.parametrize("K,nL,Q,seed", [(4, 4, (4, 0), 3), (4, 2, (3, 1), 1), (4, 6, (5, -1), 2),
                                         (3, 2, (2, 0), 8), (3, 4, (3, 1), 9)])
def test_cn_sigma_equals_fock_hamiltonian(K, nL, Q, seed):
    t, v = random_integrals(K, seed)
    ints = Integrals(t, v)
    n = 2 * K
    bL, pL, oL = fock_ops_exact(ints, list(range(nL)), "L", "cn")
    bR, pR, oR = fock_ops_exact(ints, list(range(nL, n)), "R", "cn")
    H = hamiltonian_fock(t, v).toarray()
    lay, size = psi_layout(bL, bR, Q)
    idx = _global_index(lay, bL, pL, bR, pR, nL)
    x = np.random.default_rng(seed).standard_normal(size)
    terms = cn_terms(nL, n)
    assert len(terms) == count_cn_terms(nL, n - nL)
    s = sigma_blocks(x, lay, terms, oL, oR)
    ref = H[np.ix_(idx, idx)] @ x
    assert np.abs(s - ref).max() < 1e-12 * max(1.0, np.abs(ref).max())
    Hd = heff_dense(lay, terms, oL, oR)
    assert np.abs(Hd - Hd.T).max() < 1e-12
    assert np.abs(np.diag(Hd) - heff_diagonal(lay, terms, oL, oR)).max() < 1e-12


def test_cn_and_nc_give_the_same_heff():
    """Both partitions of one cut are the same operator on the same basis."""
    K, nL, Q = 4, 4, (4, 0)
    t, v = random_integrals(K, 4)
    ints = Integrals(t, v)
    n = 2 * K
    out = []
    for kind, terms in (("nc", nc_terms(nL, n)), ("cn", cn_terms(nL, n))):
        bL, pL, oL = fock_ops_exact(ints, list(range(nL)), "L", kind)
        bR, pR, oR = fock_ops_exact(ints, list(range(nL, n)), "R", kind)
        lay, size = psi_layout(bL, bR, Q)
        out.append(heff_dense(lay, terms, oL, oR))
    assert np.abs(out[0] - out[1]).max() < 1e-12


def test_cn_term_count_is_smaller_right_of_the_middle():
    # CN at a cut with a small right block: 2 + 2n + nR(2nR - 1) terms
    assert count_cn_terms(200, 16) == 2 + 432 + 16 * 31
    assert len(cn_terms(200, 216)) == count_cn_terms(200, 16)
    assert count_cn_terms(108, 108) == 23654   # the two partitions agree at the middle


@pytest.mark.parametrize("src", ["cn", "nc"])
def test_blocking_left_cn_matches_fock_operators(src):
    K = 4
    t, v = random_integrals(K, 11)
    ints = Integrals(t, v)
    for site in range(1, K):
        bL, pL, oL = fock_ops_exact(ints, list(range(2 * site)), "L", src)
        bX, pX, oX = fock_ops_exact(ints, list(range(2 * site + 2)), "L", "cn")
        E, ch, enl = blocking_left_cn(ints, bL, oL, site, src)
        pos = np.argsort(pX)[_enlarged_index_left(E, ch, bL, pL, 2 * site)]
        assert set(enl) == set(oX)
        for k, e in enl.items():
            D = e.assemble(E, ch).to_dense()
            assert np.abs(D - oX[k].to_dense()[np.ix_(pos, pos)]).max() < 1e-12, (src, site, k)


@pytest.mark.parametrize("dst", ["cn", "nc"])
def test_blocking_right_cn_matches_fock_operators(dst):
    K = 4
    t, v = random_integrals(K, 12)
    ints = Integrals(t, v)
    n = 2 * K
    for site in range(0, K - 1):
        bR, pR, oR = fock_ops_exact(ints, list(range(2 * site + 2, n)), "R", "cn")
        bX, pX, oX = fock_ops_exact(ints, list(range(2 * site, n)), "R", dst)
        E, ch, enl = blocking_right_cn(ints, bR, oR, site, dst)
        pos = np.argsort(pX)[_enlarged_index_right(E, ch, bR, pR)]
        assert set(enl) == set(oX)
        for k, e in enl.items():
            D = e.assemble(E, ch).to_dense()
            assert np.abs(D - oX[k].to_dense()[np.ix_(pos, pos)]).max() < 1e-12, (dst, site, k)


def test_blocking_from_the_right_vacuum_in_cn_form():
    K = 3
    t, v = random_integrals(K, 13)
    ints = Integrals(t, v)
    n = 2 * K
    b0, o0 = vacuum_right_cn(ints)
    bX, pX, oX = fock_ops_exact(ints, [n - 2, n - 1], "R", "cn")
    E, ch, enl = blocking_right_cn(ints, b0, o0, K - 1, "cn")
    assert set(enl) == set(oX)
    pos = np.argsort(pX)[_enlarged_index_right(E, ch, b0, np.array([0]))]
    for k, e in enl.items():
        assert np.abs(e.assemble(E, ch).to_dense() - oX[k].to_dense()[np.ix_(pos, pos)]).max() < 1e-12, k


@pytest.mark.parametrize("K,N,two_sz,cut", [(5, 4, 0, 2), (5, 5, 1, 3), (4, 4, 0, 0), (4, 3, -1, 1)])
def test_mixed_sweeps_at_full_bond_dimension_give_fci(K, N, two_sz, cut):
    t, v = random_integrals(K, 21)
    e_fci = fci_energy(t, v, N, two_sz)
    d = PlainDMRG(t, v, N, two_sz, seed=3, dav_tol=1e-13, cut=cut)
    d.build_blocks(4 ** K)
    energies, disc = d.sweep([4 ** K] * 2)
    assert all(abs(e - e_fci) < 1e-9 for e in energies), (energies, e_fci)
    assert all(rec["energy"] - e_fci < 1e-9 for rec in d.log)   # every step, both partitions


def test_mixed_and_nc_sweeps_agree_step_by_step_when_truncated():
    """The partition changes how H_eff is assembled, not H_eff: with the same
    truncation decisions both schemes produce the same energies at each step."""
    K, N, two_sz, M = 6, 6, 0, 12
    t, v = random_integrals(K, 22)
    runs = []
    for cut in (None, 3):
        d = PlainDMRG(t, v, N, two_sz, seed=5, dav_tol=1e-13, cut=cut)
        d.build_blocks(M)
        d.sweep([M, M])
        runs.append([rec["energy"] for rec in d.log])
    # Davidson stops at |r|^2 < 1e-13; that eigenvector error enters the next
    # kept bases at first order, so later steps agree to ~1e-8, not to rounding
    diff = np.abs(np.array(runs[0]) - np.array(runs[1]))
    assert diff[:4].max() < 1e-11 and diff.max() < 1e-7, diff
