"""Pins for the oracle's sub-Hamiltonian split of sigma (Sec. II.B).

The split must (a) partition the NC terms, so the parts sum to the full
sigma; (b) keep index-symmetric and conjugate partners on one rank
(Eq. proc-def is symmetric in its two indices); (c) follow the paper's
1-based rank formula; (d) balance the terms over ranks when P << K."""

import collections

import numpy as np
import pytest

from oracle.nc import count_nc_terms, nc_terms
from oracle.sigma import nc_term_rank, proc_two, psi_layout, sigma_blocks, sigma_part, synthetic_ops
from synth import gaussian_sector_dims, mirrored_sectors, random_unit_vector


@pytest.mark.parametrize("P", [1, 2, 3, 7])
def test_parts_sum_to_full_sigma(P):
    left = gaussian_sector_dims(60, n_spatial=3, n_tot=6)
    right = mirrored_sectors(left, n_tot=6)
    bL, bR, oL, oR, _ = synthetic_ops(left, right, 6, 12, seed=4)
    lay, size = psi_layout(bL, bR, (6, 0))
    x = random_unit_vector(size, 9)
    terms = nc_terms(6, 12)
    full = sigma_blocks(x, lay, terms, oL, oR)
    parts = [sigma_part(x, lay, terms, oL, oR, r, P) for r in range(P)]
    assert np.abs(sum(parts) - full).max() <= 1e-13 * np.abs(full).max()
    if P > 1:
        assert all(np.abs(p).max() > 0 for p in parts)


def test_partners_share_a_rank():
    terms = nc_terms(10, 20)
    for P in (2, 3, 5, 8):
        for a, b in zip(terms[2::2], terms[3::2]):   # conjugate pairs of the a+/R, R/a, A/P families
            if a[0][0] in ("cd", "RL", "A"):
                assert nc_term_rank(a, P) == nc_term_rank(b, P)
        rank_of = {}
        for t in terms:
            if t[0] is not None and t[0] != "H" and t[0][0] == "B":
                rank_of.setdefault(t[0], set()).add(nc_term_rank(t, P))
        assert all(len(s) == 1 for s in rank_of.values())   # B_pq and B_qp = B_pq^T together


def test_pair_rule_is_the_papers_formula():
    for P in (2, 3, 5, 8):
        for i1 in range(1, 20):          # 1-based as printed: i <= j
            for j1 in range(i1, 20):
                p1 = ((j1 - 1) * j1 // 2 + i1 - 1) % P + 1     # the p in 1..P with p = (j-1)j/2 + i mod P
                assert proc_two(i1 - 1, j1 - 1, P) == p1 - 1
                assert proc_two(j1 - 1, i1 - 1, P) == p1 - 1


@pytest.mark.parametrize("P", [2, 4, 8])
def test_terms_balance_over_ranks_at_k108(P):
    terms = nc_terms(108, 216)
    assert len(terms) == count_nc_terms(108, 108) == 23654
    cnt = collections.Counter(nc_term_rank(t, P) for t in terms)
    mean = len(terms) / P
    assert set(cnt) == set(range(P))
    assert max(abs(c - mean) for c in cnt.values()) < 0.02 * mean


@pytest.mark.parametrize("P", [2, 3, 5])
def test_cn_parts_sum_to_full_sigma_and_use_the_large_indices(P):
    """CN partition (Eq. proc-def-cn): a two-index term is placed by its
    right-block pair, i.e. by the two larger orbital indices; the parts
    still partition the terms."""
    from oracle.cn import cn_terms
    from oracle.nc import Integrals, fock_ops_exact
    from synth import random_integrals
    K, nL = 4, 4
    t, v = random_integrals(K, 2)
    ints = Integrals(t, v)
    bL, _, oL = fock_ops_exact(ints, list(range(nL)), "L", "cn")
    bR, _, oR = fock_ops_exact(ints, list(range(nL, 2 * K)), "R", "cn")
    lay, size = psi_layout(bL, bR, (4, 0))
    x = random_unit_vector(size, 3)
    terms = cn_terms(nL, 2 * K)
    full = sigma_blocks(x, lay, terms, oL, oR)
    parts = [sigma_part(x, lay, terms, oL, oR, r, P) for r in range(P)]
    assert np.abs(sum(parts) - full).max() <= 1e-13 * np.abs(full).max()
    for term in terms:
        if term[0] is not None and term[0] != "H" and term[0][0] in ("P", "Q"):
            p, r = term[0][1], term[0][2]
            assert p >= nL and r >= nL
            assert nc_term_rank(term, P) == proc_two(p, r, P)
