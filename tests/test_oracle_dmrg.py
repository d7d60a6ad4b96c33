"""Pins of the plain DMRG and Davidson: full bond dimension reproduces FCI."""

import json
import os

import numpy as np
import pytest

from oracle.davidson import davidson
from oracle.dmrg import PlainDMRG
from oracle.fock import fci_energy
from synth import random_integrals

GOLD = os.path.join(os.path.dirname(__file__), "golden", "fci_energies.json")


def test_davidson_matches_dense_eigh():
    rng = np.random.default_rng(0)
    for n in (5, 60, 300):
        A = rng.standard_normal((n, n))
        A = A + A.T + np.diag(np.arange(n) * 0.3)
        th, x, nmv, conv = davidson(lambda v: A @ v, np.diag(A).copy(), rng.standard_normal(n),
                                    tol=1e-22, max_iter=600)
        w = np.linalg.eigvalsh(A)
        assert conv and abs(th - w[0]) < 1e-10
        assert np.linalg.norm(A @ x - th * x) < 1e-9


@pytest.mark.parametrize("K,N,s,M", [(4, 4, 0, 16), (5, 5, 1, 32), (4, 3, -1, 16)])
def test_full_m_dmrg_equals_fci(K, N, s, M):
    t, v = random_integrals(K, 7)
    d = PlainDMRG(t, v, N, s, seed=1)
    d.build_blocks(M)
    e, disc = d.sweep([M] * 2)
    ref = fci_energy(t, v, N, s)
    assert all(abs(x - ref) < 1e-9 for x in e)
    assert all(w < 1e-20 for w in disc)


def test_truncated_dmrg_is_variational_and_improves():
    t, v = random_integrals(5, 7)
    ref = fci_energy(t, v, 4, 2)
    d = PlainDMRG(t, v, 4, 2, seed=1)
    d.build_blocks(8)
    e, disc = d.sweep([8, 8, 8, 8])
    assert all(x > ref - 1e-9 for x in e)
    assert e[-1] < e[0]
    assert max(disc) > 0


def test_config1_full_m_equals_stored_fci():
    """K=8, N=8, Sz=0, seed 0, M=256: every bond is at full dimension."""
    gold = json.load(open(GOLD))["cfg1"]
    t, v = random_integrals(8, 0)
    d = PlainDMRG(t, v, 8, 0, seed=0)
    d.build_blocks(256)
    e, disc = d.sweep([256, 256])
    assert all(abs(x - gold["energy"]) < 1e-9 for x in e)


def test_wavefunction_prediction_is_exact_at_full_bond_dimension():
    """At full bond dimension every kept basis spans its whole space, so the
    previous ground state carried to the next bond (predict) is the same
    state: unit norm and Rayleigh quotient equal to the FCI energy. A wrong
    index, block or transpose in the carry breaks both."""
    from oracle.cn import mixed_terms
    from oracle.fock import fci_energy
    from oracle.sigma import sigma_blocks
    K, N, s = 5, 5, 1
    t, v = random_integrals(K, 3)
    e_fci = fci_energy(t, v, N, s)
    d = PlainDMRG(t, v, N, s, seed=2, dav_tol=1e-24, dav_max_iter=400)
    d.build_blocks(4 ** K)
    checked = 0
    for sweep in range(3):
        fwd = sweep % 2 == 0
        for i in (range(0, K - 1) if fwd else range(K - 2, -1, -1)):
            g = d.predict(i, fwd)
            if g is not None and d.prev[0] != i:
                EL, oL, ER, oR = d.enlarged(i)
                from oracle.sigma import psi_layout
                lay, size = psi_layout(EL, ER, d.Q)
                assert abs(np.linalg.norm(g) - 1.0) < 1e-10
                e = g @ sigma_blocks(g, lay, mixed_terms(i + 1, K, d.cut), oL, oR)
                assert abs(e - e_fci) < 1e-9, (sweep, i, e, e_fci)
                checked += 1
            d.step(i, fwd, 4 ** K, sweep * K + i)
    assert checked == 3 * (K - 2)
    assert all(rec["nmv"] <= 3 for rec in d.log[K - 1:])   # converged guesses after the first sweep
