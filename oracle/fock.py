"""Fock-space operators, the ab initio Hamiltonian and FCI (oracle side).

Spin orbitals: p = 2*i + sigma for spatial orbital i, sigma = 0 (alpha),
1 (beta). A Fock state is an integer whose bit p is the occupation of mode p,
ordered so that |n> = (a+_0)^n_0 (a+_1)^n_1 ... |vac> (Jordan-Wigner order =
ascending p). Then a+_p |n> = (-1)^(sum_{q<p} n_q) |n + e_p> if n_p = 0.

Hamiltonian (Appendix B, Eq. qc-hamil), chemist's notation v_ijkl = (ij|kl):
    H = sum_{ij,s} t_ij a+_{is} a_{js}
      + 1/2 sum_{ijkl,s,s'} v_ijkl a+_{is} a+_{ks'} a_{ls'} a_{js}
No nuclear-repulsion or core constant is added.

Parity status: pinned (tests/test_oracle_fci.py) against closed forms
(non-interacting energies, Hubbard dimer, two-electron first-quantised CI,
fully filled determinant) and against brute-force Fock-space products.
"""

import itertools

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla


def popcount(x):
    x = np.asarray(x, dtype=np.int64)
    c = np.zeros_like(x)
    y = x.copy()
    while np.any(y):
        c += y & 1
        y >>= 1
    return c


def qn_of_states(states):
    """(N, 2Sz) of integer Fock states (alpha = even bits, beta = odd bits)."""
    states = np.asarray(states, dtype=np.int64)
    n = popcount(states)
    amask = 0x5555555555555555 & ((1 << 62) - 1)
    na = popcount(states & amask)
    return n, 2 * na - n


def sector_states(n_modes, N, two_sz):
    """Sorted integer states of n_modes spin orbitals with N electrons, 2Sz."""
    K = n_modes // 2
    na = (N + two_sz) // 2
    nb = N - na
    if (N + two_sz) % 2 or na < 0 or nb < 0 or na > K or nb > K:
        return np.zeros(0, dtype=np.int64)
    out = []
    for ca in itertools.combinations(range(K), na):
        abits = sum(1 << (2 * i) for i in ca)
        for cb in itertools.combinations(range(K), nb):
            out.append(abits | sum(1 << (2 * i + 1) for i in cb))
    return np.array(sorted(out), dtype=np.int64)


def cre_fock(n_modes, p):
    """a+_p as a sparse (2^n x 2^n) matrix on the full Fock space."""
    dim = 1 << n_modes
    s = np.arange(dim, dtype=np.int64)
    ok = (s >> p) & 1 == 0
    src = s[ok]
    dst = src | (1 << p)
    below = src & ((1 << p) - 1)
    sign = np.where(popcount(below) % 2 == 0, 1.0, -1.0)
    return sp.csr_matrix((sign, (dst, src)), shape=(dim, dim))


def hamiltonian_fock(t, v):
    """Full-Fock-space sparse H for small K (2K <= 12 modes), by operator products."""
    K = t.shape[0]
    n = 2 * K
    c = [cre_fock(n, p) for p in range(n)]
    a = [x.T.tocsr() for x in c]
    H = sp.csr_matrix((1 << n, 1 << n))
    for i in range(K):
        for j in range(K):
            if t[i, j] != 0.0:
                for s in range(2):
                    H = H + t[i, j] * (c[2 * i + s] @ a[2 * j + s])
    for i, j, k, l in itertools.product(range(K), repeat=4):
        x = v[i, j, k, l]
        if x == 0.0:
            continue
        for s in range(2):
            for s2 in range(2):
                H = H + 0.5 * x * (c[2 * i + s] @ c[2 * k + s2] @ a[2 * l + s2] @ a[2 * j + s])
    return H.tocsr()


def _annihilator_between(states_from, states_to, p):
    """a_p restricted: maps span(states_from) -> span(states_to), sparse."""
    idx_to = {int(s): k for k, s in enumerate(states_to)}
    rows, cols, vals = [], [], []
    for k, s in enumerate(states_from):
        s = int(s)
        if (s >> p) & 1:
            d = s ^ (1 << p)
            sign = -1.0 if bin(s & ((1 << p) - 1)).count("1") % 2 else 1.0
            rows.append(idx_to[d])
            cols.append(k)
            vals.append(sign)
    return sp.csr_matrix((vals, (rows, cols)), shape=(len(states_to), len(states_from)))


def excitation_ops(K, N, two_sz):
    """E^s_ij = a+_{is} a_{js} restricted to the (N, 2Sz) sector, for s in {0,1}."""
    n = 2 * K
    st = sector_states(n, N, two_sz)
    st_a = sector_states(n, N - 1, two_sz - 1)  # after removing an alpha
    st_b = sector_states(n, N - 1, two_sz + 1)  # after removing a beta
    E = {}
    for s, lower in ((0, st_a), (1, st_b)):
        ann = [_annihilator_between(st, lower, 2 * j + s) for j in range(K)]
        for i in range(K):
            cre = ann[i].T.tocsr()
            for j in range(K):
                E[(s, i, j)] = (cre @ ann[j]).tocsr()
    return st, E


def hamiltonian_sector(t, v, N, two_sz):
    """Sparse H restricted to the (N, 2Sz) sector, via spin-summed excitations:
    H = sum t_ij E_ij + 1/2 sum v_ijkl (E_ij E_kl - delta_jk E_il)."""
    K = t.shape[0]
    st, Es = excitation_ops(K, N, two_sz)
    E = {(i, j): (Es[(0, i, j)] + Es[(1, i, j)]).tocsr() for i in range(K) for j in range(K)}
    dim = len(st)
    H = sp.csr_matrix((dim, dim))
    for i in range(K):
        for j in range(K):
            H = H + t[i, j] * E[(i, j)]
    for i in range(K):
        for j in range(K):
            W = sp.csr_matrix((dim, dim))
            for k in range(K):
                for l in range(K):
                    if v[i, j, k, l] != 0.0:
                        W = W + v[i, j, k, l] * E[(k, l)]
            H = H + 0.5 * (E[(i, j)] @ W)
    for i in range(K):
        for l in range(K):
            x = sum(v[i, j, j, l] for j in range(K))
            if x != 0.0:
                H = H - 0.5 * x * E[(i, l)]
    return st, H.tocsr()


def fci_energy(t, v, N, two_sz, dense_limit=6000):
    """Lowest eigenvalue of H in the (N, 2Sz) sector (dense eigh up to dense_limit)."""
    st, H = hamiltonian_sector(t, v, N, two_sz)
    if H.shape[0] <= dense_limit:
        return float(np.linalg.eigvalsh(H.toarray())[0])
    w = spla.eigsh(H, k=1, which="SA", tol=1e-13)[0]
    return float(w[0])
