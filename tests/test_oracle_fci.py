"""Pins of the oracle FCI (Eq. qc-hamil) against closed forms and brute force."""

import itertools

import numpy as np
import pytest

from oracle.fock import fci_energy, hamiltonian_fock, hamiltonian_sector, sector_states
from synth import random_integrals


def test_hubbard_dimer_closed_form():
    # two sites, hopping -tau, on-site U: E0 = U/2 - sqrt(U^2/4 + 4 tau^2)
    for tau, U in ((1.0, 4.0), (0.7, 1.3), (1.0, 0.0)):
        t = np.array([[0.0, -tau], [-tau, 0.0]])
        v = np.zeros((2, 2, 2, 2))
        v[0, 0, 0, 0] = v[1, 1, 1, 1] = U
        assert abs(fci_energy(t, v, 2, 0) - (U / 2 - np.sqrt(U * U / 4 + 4 * tau * tau))) < 1e-12


def test_noninteracting_is_sum_of_orbital_energies():
    t, _ = random_integrals(5, 3)
    v = np.zeros((5,) * 4)
    eps = np.linalg.eigvalsh(t)
    for N, s in ((4, 0), (5, 1), (3, -1), (6, 2)):
        na, nb = (N + s) // 2, (N - s) // 2
        ref = eps[:na].sum() + eps[:nb].sum()
        assert abs(fci_energy(t, v, N, s) - ref) < 1e-11


def test_two_electron_first_quantised_ci():
    # N=2, Sz=0: H[(i,j),(k,l)] = t_ik d_jl + d_ik t_jl + (ik|jl), alpha electron
    # in i/k, beta electron in j/l (chemist's notation)
    K = 4
    t, v = random_integrals(K, 9)
    H = np.zeros((K * K, K * K))
    for i, j, k, l in itertools.product(range(K), repeat=4):
        H[i * K + j, k * K + l] = t[i, k] * (j == l) + (i == k) * t[j, l] + v[i, k, j, l]
    assert abs(fci_energy(t, v, 2, 0) - np.linalg.eigvalsh(H)[0]) < 1e-11


def test_filled_determinant_closed_form():
    K = 4
    t, v = random_integrals(K, 4)
    ref = 2 * np.trace(t) + sum(2 * v[i, i, j, j] - v[i, j, j, i] for i in range(K) for j in range(K))
    assert abs(fci_energy(t, v, 2 * K, 0) - ref) < 1e-11


def test_sector_matrix_equals_fock_products_and_is_hermitian():
    t, v = random_integrals(3, 0)
    Hf = hamiltonian_fock(t, v).toarray()
    assert np.abs(Hf - Hf.T).max() < 1e-13
    for N, s in ((3, 1), (2, 0), (4, -2)):
        st, Hs = hamiltonian_sector(t, v, N, s)
        assert np.abs(Hf[np.ix_(st, st)] - Hs.toarray()).max() < 1e-13
    # H conserves N and Sz: no element couples different sectors
    from oracle.fock import qn_of_states
    n, sz = qn_of_states(np.arange(64))
    rows, cols = np.nonzero(np.abs(Hf) > 1e-14)
    assert np.all(n[rows] == n[cols]) and np.all(sz[rows] == sz[cols])


def test_sector_sizes():
    assert len(sector_states(16, 8, 0)) == 4900  # C(8,4)^2
    assert len(sector_states(16, 9, 1)) == 70 * 56
