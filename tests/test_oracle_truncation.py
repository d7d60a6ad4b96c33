"""Pins for the oracle's truncated (M below full) DMRG blocks.

Every renormalized block of the oracle stands for a set of orthonormal
states of the Fock space of its modes: composing the kept columns U of each
blocking step (Eq. op-trans) with the product states of block x site gives
those states explicitly. Because each enlarged operator is a sum of (whole
block operator) x (site operator), the renormalized operators must equal
the exact Fock-space operators projected on those states, V^T O V, at any
bond dimension; and the energy of a two-site step must equal the lowest
eigenvalue of the Fock-space Hamiltonian projected on L x site x site x R.
A dropped term, a wrong sign or a transposed U in blocking or
transformation breaks one of these.
"""

import numpy as np
import scipy.sparse as sp

from oracle.blocks import enlarged_left, enlarged_right
from oracle.dmrg import PlainDMRG
from oracle.fock import hamiltonian_fock, qn_of_states
from oracle.nc import fock_ops_exact
from synth import random_integrals

K, N, TWO_SZ, M = 5, 4, 2, 8


def _raw(D, perm):
    """Matrix over the sector-ordered basis -> matrix over raw Fock states."""
    out = np.zeros((len(perm), len(perm)))
    out[np.ix_(perm, perm)] = D
    return out


def _compose(prev, basis_prev, nb, U, chunks, E, left, shift):
    """Raw Fock vectors (columns) of the kept states nb of block x site."""
    dim = prev.shape[0] * 4
    W = np.zeros((dim, E.total))
    for Q in E.qs:
        base = E.offsets[E.index[Q]]
        for qb, ns, off in chunks[Q]:
            i0 = basis_prev.offsets[basis_prev.index[qb]]
            for a in range(basis_prev.dim(qb)):
                col = prev[:, i0 + a]
                for raw in np.nonzero(col)[0]:
                    r = (raw | (ns << shift)) if left else (ns | (raw << 2))
                    W[r, base + off + a] = col[raw]
    V = np.zeros((dim, nb.total))
    for Q in nb.qs:
        rows = slice(E.offsets[E.index[Q]], E.offsets[E.index[Q]] + E.dim(Q))
        V[:, nb.offsets[nb.index[Q]]:nb.offsets[nb.index[Q]] + nb.dim(Q)] = W[:, rows] @ U[Q]
    return V


def _right_states(d):
    vec = {K: np.ones((1, 1))}
    for j in range(K - 1, 0, -1):
        if j not in d.UR:
            break
        bprev = d.R[j + 1][0]
        E, ch = enlarged_right(bprev)
        vec[j] = _compose(vec[j + 1], bprev, d.R[j][0], d.UR[j], ch, E, False, 0)
    return vec


def _left_states(d):
    vec = {0: np.ones((1, 1))}
    for i in range(1, K):
        if i not in d.UL:
            break
        bprev = d.L[i - 1][0]
        E, ch = enlarged_left(bprev)
        vec[i] = _compose(vec[i - 1], bprev, d.L[i][0], d.UL[i], ch, E, True, 2 * (i - 1))
    return vec


def _check_block(d, vecs, blocks, modes_of, side):
    for j, V in vecs.items():
        if j in (0, K) or j not in blocks:
            continue
        basis, ops = blocks[j]
        assert np.abs(V.T @ V - np.eye(V.shape[1])).max() < 1e-12
        kind = "nc" if j <= d.cut else "cn"   # block of j left orbitals / starting at orbital j
        _, perm, exact = fock_ops_exact(d.ints, modes_of(j), side, kind)
        assert set(ops) == set(exact)
        for key, op in ops.items():
            ref = V.T @ _raw(exact[key].to_dense(), perm) @ V
            got = op.to_dense()
            assert got.shape == ref.shape
            assert np.abs(got - ref).max() < 1e-11, (side, j, key)


def test_initial_right_blocks_are_projections():
    t, v = random_integrals(K, 7)
    d = PlainDMRG(t, v, N, TWO_SZ, seed=1)
    d.build_blocks(M)
    vecs = _right_states(d)
    assert any(d.R[j][0].total < 4 ** (K - j) for j in range(1, K))  # truncated
    _check_block(d, vecs, d.R, lambda j: list(range(2 * j, 2 * K)), "R")


def test_swept_blocks_are_projections():
    t, v = random_integrals(K, 7)
    d = PlainDMRG(t, v, N, TWO_SZ, seed=1, dav_tol=1e-12)
    d.build_blocks(M)
    d.sweep([M, M])
    _check_block(d, _left_states(d), d.L, lambda i: list(range(0, 2 * i)), "L")
    _check_block(d, _right_states(d), d.R, lambda j: list(range(2 * j, 2 * K)), "R")


def test_mixed_nc_cn_blocks_are_projections():
    """Mixed NC/CN (cut after orbital 2): blocks on both sides of the cut,
    including the ones made by the normal-to-complementary transformation,
    are exact projections of their Fock-space operators."""
    t, v = random_integrals(K, 7)
    d = PlainDMRG(t, v, N, TWO_SZ, seed=1, dav_tol=1e-12, cut=2)
    d.build_blocks(M)
    _check_block(d, _right_states(d), d.R, lambda j: list(range(2 * j, 2 * K)), "R")
    d.sweep([M, M])
    assert {k[0] for k in d.L[4][1] if isinstance(k, tuple)} == {"cd", "RL", "P", "Q"}
    assert {k[0] for k in d.R[4][1] if isinstance(k, tuple)} == {"d", "RR", "A", "B"}
    _check_block(d, _left_states(d), d.L, lambda i: list(range(0, 2 * i)), "L")
    _check_block(d, _right_states(d), d.R, lambda j: list(range(2 * j, 2 * K)), "R")


def test_step_energy_is_projected_fock_ground_state():
    t, v = random_integrals(K, 7)
    d = PlainDMRG(t, v, N, TWO_SZ, seed=1, dav_tol=1e-13)
    d.build_blocks(M)
    R2 = _right_states(d)[2]
    # bond 0: (vacuum) x site 0 x site 1 x R[2]; raw = n0 | n1 << 2 | r << 4
    cols = []
    for n0 in range(4):
        for n1 in range(4):
            for k in range(R2.shape[1]):
                c = np.zeros(1 << (2 * K))
                for raw in np.nonzero(R2[:, k])[0]:
                    c[n0 | (n1 << 2) | (raw << 4)] = R2[raw, k]
                cols.append(c)
    P = np.array(cols).T
    nq, sq = qn_of_states(np.arange(1 << (2 * K)))
    sector = (nq == N) & (sq == TWO_SZ)
    keep = np.abs(P[~sector]).sum(axis=0) < 1e-14  # states inside the target sector
    P = P[:, keep]
    H = hamiltonian_fock(t, v)
    Hp = P.T @ (sp.csr_matrix(H) @ P)
    e_ref = np.linalg.eigvalsh(0.5 * (Hp + Hp.T))[0]
    EL, oL, ER, oR = d.enlarged(0)
    th = d.solve(0, 0, EL, oL, ER, oR)[0]
    assert abs(th - e_ref) < 1e-10, (th, e_ref)


def test_noise_and_keep_one_per_q_keep_blocks_exact_projections():
    """With perturbative noise and one kept state per quantum number, the
    renormalized operators are still exact projections on orthonormal states,
    every psi block's left sector survives each forward step, and energies stay
    variational."""
    from oracle.fock import fci_energy
    t, v = random_integrals(K, 7)
    d = PlainDMRG(t, v, N, TWO_SZ, seed=1, dav_tol=1e-12, noise=1e-2, keep_one_per_q=True)
    d.build_blocks(6)
    e, disc = d.sweep([6, 6])
    assert all(x > fci_energy(t, v, N, TWO_SZ) - 1e-9 for x in e)
    _check_block(d, _left_states(d), d.L, lambda i: list(range(0, 2 * i)), "L")
    _check_block(d, _right_states(d), d.R, lambda j: list(range(2 * j, 2 * K)), "R")
    # one step with M=1: every left sector of the two-site psi still keeps a state
    d2 = PlainDMRG(t, v, N, TWO_SZ, seed=1, dav_tol=1e-12, noise=1e-2, keep_one_per_q=True)
    d2.build_blocks(6)
    EL, oL, ER, oR = d2.enlarged(0)
    th, x, layout, nmv, conv = d2.solve(0, 0, EL, oL, ER, oR)
    kept, svd, disc = d2.decimate(d2.perturb(x, 0), layout, 1, True)
    assert set(kept) == {qL for qL, qR, mL, mR, off in layout if min(mL, mR) > 0}


def test_perturb_is_seeded_unit_norm_and_off_without_noise():
    t, v = random_integrals(K, 7)
    d = PlainDMRG(t, v, N, TWO_SZ, seed=1, noise=1e-3)
    x = np.random.default_rng(0).standard_normal(50)
    x /= np.linalg.norm(x)
    y1, y2 = d.perturb(x, 7), d.perturb(x, 7)
    assert np.array_equal(y1, y2) and abs(np.linalg.norm(y1) - 1.0) < 1e-14
    assert 0 < min(np.linalg.norm(y1 - x), np.linalg.norm(y1 + x)) < 3e-3   # up to the sign of x
    assert not np.array_equal(d.perturb(x, 8), y1)
    d0 = PlainDMRG(t, v, N, TWO_SZ, seed=1)
    assert d0.perturb(x, 7) is x
