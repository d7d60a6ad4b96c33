"""U(1)xU(1) normal/complementary (NC) decomposition, blocking and
transformation of renormalized operators (oracle side).

The paper prints the NC left-right decomposition in SU(2) form (Appendix B,
Eq. h-nc with the operator definitions of Eq. op-def and the index symmetry
of Eq. index-sym). With only N and Sz conserved, the same decomposition in
spin orbitals p = 2i + sigma (L modes before R modes in Jordan-Wigner order,
"X (x) Y" meaning the operator product X*Y) reads

  H = H_L (x) 1 + 1 (x) H_R
    + sum_{p in L} ( a+_p (x) R^R_p  -  a_p (x) (R^R_p)^T )
    + sum_{p in R} ( (R^L_p)^T (x) a_p  -  R^L_p (x) a+_p )
    + sum_{p<r in L} ( A_pr (x) P_pr + A_pr^T (x) P_pr^T )
    + sum_{p,q in L} B_pq (x) Q_pq

  R^R_p = sum_{q in R} t_pq a_q + sum_{q,r,s in R} v_pqrs a+_r a_s a_q
  R^L_p = sum_{q,r,s in L} v_pqrs a+_r a_s a_q     (cross one-body terms live in R^R)
  A_pr = a+_p a+_r,   P_pr = sum_{q,s in R} v_pqrs a_s a_q
  B_pq = a+_p a_q,    Q_pq = sum_{r,s in R} (v_pqrs - v_psrq) a+_r a_s

with spin-orbital integrals t_pq = t_ij d(sp,sq) and
v_pqrs = (ij|kl) d(sp,sq) d(sr,ss). Index symmetry (Eq. index-sym, U(1)
form): A_rp = -A_pr, P_rp = -P_pr, B_qp = B_pq^T, Q_qp = Q_pq^T, so only
p<r (A, P) and p<=q (B, Q) are stored.

Matrix form in a product basis |l>|r> = c_l c_r |0>:
  <l'r'| X (x) Y |lr> = (-1)^(|Y| N(l)) X[l',l] Y[r',r].

Blocking (Eq. blocked-ops) adds one spatial orbital (a "site") to a block.
Every enlarged operator is kept as a sum of products (block op) (x) (4x4 site
matrix); the formulas for each operator kind are in blocking_left /
blocking_right below, derived by splitting each second-quantized string into
its block part and its site part. Transformation (Eq. op-trans) is
U^T O U per sector pair.

Parity status: pinned (tests/test_oracle_nc.py) - the decomposition against
the Fock-space Hamiltonian, every blocked operator against its Fock-space
matrix, and the transformation through DMRG at full bond dimension = FCI.
"""

import itertools

import numpy as np

from .blocks import (Basis, BlockOp, SITE_N, SITE_Q, enlarged_left,
                     enlarged_right, qadd, site_basis, site_cre)
from .fock import cre_fock, qn_of_states


def spin(p):
    return 1 if p % 2 == 0 else -1


class Integrals:
    """Spin-orbital view of spatial integrals (t, v)."""

    def __init__(self, t, v):
        self.t = np.asarray(t, dtype=np.float64)
        self.v = np.asarray(v, dtype=np.float64)
        self.K = self.t.shape[0]
        self.n = 2 * self.K

    def tso(self, p, q):
        return self.t[p // 2, q // 2] if p % 2 == q % 2 else 0.0

    def vso(self, p, q, r, s):
        if p % 2 != q % 2 or r % 2 != s % 2:
            return 0.0
        return self.v[p // 2, q // 2, r // 2, s // 2]


# ------------------------------------------------------------------ NC terms
def nc_terms(nL, n):
    """Canonical NC term list for L = modes [0, nL), R = modes [nL, n).

    Each term is (left_key, left_T, right_key, right_T, coef); key None means
    the identity. Keys: 'H'; ('cd', p) = a+_p; ('RL', p); ('A', p, r);
    ('B', p, q) on the left; 'H'; ('d', p) = a_p; ('RR', p); ('P', p, r);
    ('Q', p, q) on the right. Count: 2 + 4 nL' + ... (see count_nc_terms).
    """
    T = [("H", False, None, False, 1.0), (None, False, "H", False, 1.0)]
    for p in range(nL):
        T.append((("cd", p), False, ("RR", p), False, 1.0))
        T.append((("cd", p), True, ("RR", p), True, -1.0))
    for p in range(nL, n):
        T.append((("RL", p), True, ("d", p), False, 1.0))
        T.append((("RL", p), False, ("d", p), True, -1.0))
    for p in range(nL):
        for r in range(p + 1, nL):
            T.append((("A", p, r), False, ("P", p, r), False, 1.0))
            T.append((("A", p, r), True, ("P", p, r), True, 1.0))
    for p in range(nL):
        for q in range(nL):
            if p <= q:
                T.append((("B", p, q), False, ("Q", p, q), False, 1.0))
            else:
                T.append((("B", q, p), True, ("Q", q, p), True, 1.0))
    return T


def count_nc_terms(nL, nR):
    return 2 + 2 * nL + 2 * nR + nL * (nL - 1) + nL * nL


def right_parity(key):
    if key is None or key == "H":
        return 0
    return 1 if key[0] in ("d", "RR", "cd", "RL") else 0


# ------------------------------------------------- exact Fock-space operators
def fock_block_basis(modes):
    """Sector-ordered basis of the full Fock space of `modes` (consecutive,
    starting at an even mode). Returns (Basis, perm) where perm[k] is the local
    integer state of basis index k."""
    nm = len(modes)
    states = np.arange(1 << nm, dtype=np.int64)
    N, S = qn_of_states(states)
    # local bit 0 is mode modes[0]; alpha/beta follow the global parity of the
    # mode, which is the local parity because modes[0] is even.
    keys = sorted(range(len(states)), key=lambda k: (N[k], S[k], states[k]))
    perm = states[keys]
    secs = {}
    for k in keys:
        q = (int(N[k]), int(S[k]))
        secs[q] = secs.get(q, 0) + 1
    return Basis(list(secs.items())), perm


def fock_ops_exact(ints, modes, side, kind="nc"):
    """Exact matrices of all operators of a block holding `modes`, in its
    sector-ordered full Fock basis (for pins; small blocks only). side 'L'
    keeps a+_p (p in modes) and R^L_p (p outside), side 'R' keeps a_p and
    R^R_p; the two-index operators are the normal A, B over `modes` for a
    left NC or right CN block, else the complementary P, Q over the modes
    outside (kind 'nc' or 'cn', see cn.py)."""
    nm = len(modes)
    m0 = modes[0]
    basis, perm = fock_block_basis(modes)
    c = [cre_fock(nm, k).toarray()[np.ix_(perm, perm)] for k in range(nm)]
    a = [x.T for x in c]
    loc = lambda p: p - m0
    inside = set(modes)
    n = ints.n

    def op(mat, dq):
        return BlockOp.from_dense(mat, dq, basis)

    ops = {}
    H = np.zeros((1 << nm, 1 << nm))
    for p in modes:
        for q in modes:
            H += ints.tso(p, q) * c[loc(p)] @ a[loc(q)]
    for p, q, r, s in itertools.product(modes, repeat=4):
        x = ints.vso(p, q, r, s)
        if x != 0.0:
            H += 0.5 * x * c[loc(p)] @ c[loc(r)] @ a[loc(s)] @ a[loc(q)]
    ops["H"] = op(H, (0, 0))
    others = [p for p in range(n) if p not in inside]
    if side == "L":
        for p in modes:
            ops[("cd", p)] = op(c[loc(p)], (1, spin(p)))
        for p in others:
            R = np.zeros_like(H)
            for q, r, s in itertools.product(modes, repeat=3):
                x = ints.vso(p, q, r, s)
                if x != 0.0:
                    R += x * c[loc(r)] @ a[loc(s)] @ a[loc(q)]
            ops[("RL", p)] = op(R, (-1, -spin(p)))
    else:
        for p in modes:
            ops[("d", p)] = op(a[loc(p)], (-1, -spin(p)))
        for p in others:
            R = np.zeros_like(H)
            for q in modes:
                R += ints.tso(p, q) * a[loc(q)]
            for q, r, s in itertools.product(modes, repeat=3):
                x = ints.vso(p, q, r, s)
                if x != 0.0:
                    R += x * c[loc(r)] @ a[loc(s)] @ a[loc(q)]
            ops[("RR", p)] = op(R, (-1, -spin(p)))
    if (side, kind) in (("L", "nc"), ("R", "cn")):
        for p in modes:
            for r in modes:
                if p < r:
                    ops[("A", p, r)] = op(c[loc(p)] @ c[loc(r)], (2, spin(p) + spin(r)))
                if p <= r:
                    ops[("B", p, r)] = op(c[loc(p)] @ a[loc(r)], (0, spin(p) - spin(r)))
    else:
        for p in others:
            for r in others:
                if p < r:
                    P = np.zeros_like(H)
                    for q, s in itertools.product(modes, repeat=2):
                        x = ints.vso(p, q, r, s)
                        if x != 0.0:
                            P += x * a[loc(s)] @ a[loc(q)]
                    ops[("P", p, r)] = op(P, (-2, -spin(p) - spin(r)))
                if p <= r:
                    Q = np.zeros_like(H)
                    for rr, s in itertools.product(modes, repeat=2):
                        x = ints.vso(p, r, rr, s) - ints.vso(p, s, rr, r)
                        if x != 0.0:
                            Q += x * c[loc(rr)] @ a[loc(s)]
                    ops[("Q", p, r)] = op(Q, (0, -(spin(p) - spin(r))))
    return basis, perm, ops


# ------------------------------------------------------------- site operators
SC = [site_cre(0), site_cre(1)]
SA = [SC[0].T, SC[1].T]
I4 = np.eye(4)


def site_mats(site):
    """Dict mode -> (a+, a) 4x4 matrices for the two modes of spatial `site`."""
    return {2 * site: (SC[0], SA[0]), 2 * site + 1: (SC[1], SA[1])}


def site_R(ints, p, site, one_body):
    """R_p restricted to the site's modes: [sum t_pq a_q] + sum v_pqrs a+_r a_s a_q."""
    sm = site_mats(site)
    m = np.zeros((4, 4))
    if one_body:
        for q, (cq, aq) in sm.items():
            m += ints.tso(p, q) * aq
    for q, r, s in itertools.product(sm, repeat=3):
        x = ints.vso(p, q, r, s)
        if x != 0.0:
            m += x * sm[r][0] @ sm[s][1] @ sm[q][1]
    return m


def site_P(ints, p, r, site):
    sm = site_mats(site)
    m = np.zeros((4, 4))
    for q, s in itertools.product(sm, repeat=2):
        x = ints.vso(p, q, r, s)
        if x != 0.0:
            m += x * sm[s][1] @ sm[q][1]
    return m


def site_Q(ints, p, q, site):
    sm = site_mats(site)
    m = np.zeros((4, 4))
    for r, s in itertools.product(sm, repeat=2):
        x = ints.vso(p, q, r, s) - ints.vso(p, s, r, q)
        if x != 0.0:
            m += x * sm[r][0] @ sm[s][1]
    return m


def site_H(ints, site):
    sm = site_mats(site)
    m = np.zeros((4, 4))
    for p, q in itertools.product(sm, repeat=2):
        m += ints.tso(p, q) * sm[p][0] @ sm[q][1]
    for p, q, r, s in itertools.product(sm, repeat=4):
        x = ints.vso(p, q, r, s)
        if x != 0.0:
            m += 0.5 * x * sm[p][0] @ sm[r][0] @ sm[s][1] @ sm[q][1]
    return m


def site_shift(mat):
    """Quantum-number shift and parity of a 4x4 site matrix (must be definite)."""
    nz = np.argwhere(np.abs(mat) > 0)
    if len(nz) == 0:
        return None
    dqs = {(SITE_Q[i][0] - SITE_Q[j][0], SITE_Q[i][1] - SITE_Q[j][1]) for i, j in nz}
    assert len(dqs) == 1, dqs
    return dqs.pop()


# ------------------------------------------------------------ enlarged ops
class EnlOp:
    """Operator on an enlarged block as sum_{n',n} X_{n'n} (x) |n'><n| (left
    enlarged, side 'L': block then site) or |n'><n| (x) X_{n'n} (side 'R')."""

    def __init__(self, side, dq, bblk):
        self.side = side
        self.dq = tuple(dq)
        self.bblk = bblk
        self.units = {}

    def add(self, c, bop, smat):
        """Add c * bop (x) smat (side L) or c * smat (x) bop (side R); bop None = 1."""
        if c == 0.0:
            return self
        if bop is None:
            bop = BlockOp.identity(self.bblk)
        for nn, n in np.argwhere(np.abs(smat) > 0):
            dsite = (SITE_Q[nn][0] - SITE_Q[n][0], SITE_Q[nn][1] - SITE_Q[n][1])
            assert (bop.dq[0] + dsite[0], bop.dq[1] + dsite[1]) == self.dq, (bop.dq, dsite, self.dq)
            key = (int(nn), int(n))
            if key not in self.units:
                self.units[key] = BlockOp.zeros(bop.dq, self.bblk)
            self.units[key].axpy(c * smat[nn, n], bop)
        return self

    def assemble(self, E, chunks):
        """Dense sector blocks over the enlarged basis E."""
        out = BlockOp.zeros(self.dq, E)
        cindex = {Q: {(qb, n): off for qb, n, off in lst} for Q, lst in chunks.items()}
        for (nn, n), X in self.units.items():
            for Q in E.qs:
                Qo = qadd(Q, self.dq)
                if not E.has(Qo):
                    continue
                for qb, n_in, off_in in chunks[Q]:
                    if n_in != n or qb not in X.blocks:
                        continue
                    qbo = qadd(qb, X.dq)
                    off_out = cindex[Qo].get((qbo, nn))
                    if off_out is None:
                        continue
                    blk = X.blocks[qb]
                    if self.side == "L":
                        par = (SITE_N[nn] - SITE_N[n]) % 2
                        sign = -1.0 if (par and qb[0] % 2) else 1.0
                    else:
                        sign = -1.0 if (X.parity and SITE_N[n] % 2) else 1.0
                    out.blocks[Q][off_out:off_out + blk.shape[0],
                                  off_in:off_in + blk.shape[1]] += sign * blk
        return out


def _getB(ops, p, q):
    return ops[("B", p, q)] if p <= q else ops[("B", q, p)].T()


def _getQ(ops, p, q):
    return ops[("Q", p, q)] if p <= q else ops[("Q", q, p)].T()


def _weighted(terms, dq, basis):
    """sum c * op over (c, op) pairs as one BlockOp."""
    acc = BlockOp.zeros(dq, basis)
    for c, o in terms:
        if c != 0.0:
            acc.axpy(c, o)
    return acc


def blocking_left(ints, bL, opsL, site):
    """Enlarged operators of L x site. L holds modes [0, 2*site). Returns
    (E, chunks, enl_ops) with enl_ops keyed like a left block of modes
    [0, 2*site+2): 'H', ('cd',p), ('A',p,r), ('B',p,q), ('RL',p) for p >= 2*site+2."""
    n = ints.n
    Lm = list(range(0, 2 * site))
    Sm = [2 * site, 2 * site + 1]
    sm = site_mats(site)
    E, chunks = enlarged_left(bL)
    eo = {}

    def new(dq):
        return EnlOp("L", dq, bL)

    for p in Lm:
        eo[("cd", p)] = new((1, spin(p))).add(1.0, opsL[("cd", p)], I4)
    for p in Sm:
        eo[("cd", p)] = new((1, spin(p))).add(1.0, None, sm[p][0])
    newm = Lm + Sm
    for p in newm:
        for r in newm:
            if p < r:
                e = new((2, spin(p) + spin(r)))
                if r in Lm:
                    e.add(1.0, opsL[("A", p, r)], I4)
                elif p in Lm:
                    e.add(1.0, opsL[("cd", p)], sm[r][0])
                else:
                    e.add(1.0, None, sm[p][0] @ sm[r][0])
                eo[("A", p, r)] = e
            if p <= r:
                e = new((0, spin(p) - spin(r)))
                if r in Lm:
                    e.add(1.0, opsL[("B", p, r)], I4)
                elif p in Lm:
                    e.add(1.0, opsL[("cd", p)], sm[r][1])
                else:
                    e.add(1.0, None, sm[p][0] @ sm[r][1])
                eo[("B", p, r)] = e
    # H of L x s: NC decomposition over (L | s)
    e = new((0, 0))
    e.add(1.0, opsL["H"], I4)
    e.add(1.0, None, site_H(ints, site))
    for p in Lm:
        Rs = site_R(ints, p, site, one_body=True)
        e.add(1.0, opsL[("cd", p)], Rs)
        e.add(-1.0, opsL[("cd", p)].T(), Rs.T)
    for p in Sm:
        e.add(1.0, opsL[("RL", p)].T(), sm[p][1])
        e.add(-1.0, opsL[("RL", p)], sm[p][0])
    for p in Lm:
        for r in Lm:
            if p < r:
                Ps = site_P(ints, p, r, site)
                e.add(1.0, opsL[("A", p, r)], Ps)
                e.add(1.0, opsL[("A", p, r)].T(), Ps.T)
    for p in Lm:
        for q in Lm:
            e.add(1.0, _getB(opsL, p, q), site_Q(ints, p, q, site))
    eo["H"] = e
    # R^L_p for p right of the enlarged block
    for p in range(2 * site + 2, n):
        e = new((-1, -spin(p)))
        e.add(1.0, opsL[("RL", p)], I4)
        e.add(1.0, None, site_R(ints, p, site, one_body=False))
        for x in Sm:
            dqB = (0, -spin(p) + spin(x))
            X = _weighted([(ints.vso(p, x, r, y) - ints.vso(p, y, r, x), _getB(opsL, r, y))
                           for r in Lm for y in Lm if (0, spin(r) - spin(y)) == dqB], dqB, bL)
            e.add(1.0, X, sm[x][1])
        for r in Sm:  # case r on site: (a_s a_q)_L (x) a+_r
            dqA = (-2, -spin(p) - spin(r))
            terms = []
            for q in Lm:
                for s in Lm:
                    x = ints.vso(p, q, r, s)
                    if x == 0.0 or q == s:
                        continue
                    if q < s:
                        terms.append((x, opsL[("A", q, s)].T()))
                    else:
                        terms.append((-x, opsL[("A", s, q)].T()))
            e.add(1.0, _weighted(terms, dqA, bL), sm[r][0])
        for s in Lm:  # q, r on site; s in L: -a_s (x) a+_r a_q
            m = np.zeros((4, 4))
            for q in Sm:
                for r in Sm:
                    m += ints.vso(p, q, r, s) * sm[r][0] @ sm[q][1]
            if np.any(m):
                e.add(-1.0, opsL[("cd", s)].T(), m)
        for r in Lm:  # q, s on site; r in L: a+_r (x) a_s a_q
            m = np.zeros((4, 4))
            for q in Sm:
                for s in Sm:
                    m += ints.vso(p, q, r, s) * sm[s][1] @ sm[q][1]
            if np.any(m):
                e.add(1.0, opsL[("cd", r)], m)
        for q in Lm:  # r, s on site; q in L: a_q (x) a+_r a_s
            m = np.zeros((4, 4))
            for r in Sm:
                for s in Sm:
                    m += ints.vso(p, q, r, s) * sm[r][0] @ sm[s][1]
            if np.any(m):
                e.add(1.0, opsL[("cd", q)].T(), m)
        eo[("RL", p)] = e
    return E, chunks, eo


def blocking_right(ints, bR, opsR, site):
    """Enlarged operators of site x R. R holds modes [2*site+2, n). Returns
    (E, chunks, enl_ops) keyed like a right block of modes [2*site, n):
    'H', ('d',p), ('RR',p), ('P',p,r), ('Q',p,q) for p, q, r < 2*site."""
    n = ints.n
    Rm = list(range(2 * site + 2, n))
    Sm = [2 * site, 2 * site + 1]
    sm = site_mats(site)
    E, chunks = enlarged_right(bR)
    eo = {}

    def new(dq):
        return EnlOp("R", dq, bR)

    for p in Sm:
        eo[("d", p)] = new((-1, -spin(p))).add(1.0, None, sm[p][1])
    for p in Rm:
        eo[("d", p)] = new((-1, -spin(p))).add(1.0, opsR[("d", p)], I4)
    # H of s x R: NC decomposition over (s | R)
    e = new((0, 0))
    e.add(1.0, None, site_H(ints, site))
    e.add(1.0, opsR["H"], I4)
    for p in Sm:
        e.add(1.0, opsR[("RR", p)], sm[p][0])
        e.add(-1.0, opsR[("RR", p)].T(), sm[p][1])
    for p in Rm:
        Rs = site_R(ints, p, site, one_body=False)
        e.add(1.0, opsR[("d", p)], Rs.T)
        e.add(-1.0, opsR[("d", p)].T(), Rs)
    p, r = Sm
    A = sm[p][0] @ sm[r][0]
    e.add(1.0, opsR[("P", p, r)], A)
    e.add(1.0, opsR[("P", p, r)].T(), A.T)
    for p in Sm:
        for q in Sm:
            e.add(1.0, _getQ(opsR, p, q), sm[p][0] @ sm[q][1])
    eo["H"] = e
    left = list(range(0, 2 * site))
    for p in left:
        e = new((-1, -spin(p)))
        e.add(1.0, opsR[("RR", p)], I4)
        e.add(1.0, None, site_R(ints, p, site, one_body=True))
        for x in Sm:
            e.add(1.0, _getQ(opsR, p, x), sm[x][1])
            e.add(1.0, opsR[("P", p, x)], sm[x][0])
        for y in Rm:
            m1 = np.zeros((4, 4))  # q, r on site, s = y in R: -(a+_r a_q) (x) a_y
            m2 = np.zeros((4, 4))  # q, s on site, r = y in R: (a_s a_q) (x) a+_y
            m3 = np.zeros((4, 4))  # r, s on site, q = y in R: (a+_r a_s) (x) a_y
            for u in Sm:
                for w in Sm:
                    m1 += ints.vso(p, u, w, y) * sm[w][0] @ sm[u][1]
                    m2 += ints.vso(p, u, y, w) * sm[w][1] @ sm[u][1]
                    m3 += ints.vso(p, y, u, w) * sm[u][0] @ sm[w][1]
            e.add(-1.0, opsR[("d", y)], m1)
            e.add(1.0, opsR[("d", y)].T(), m2)
            e.add(1.0, opsR[("d", y)], m3)
        eo[("RR", p)] = e
    for p in left:
        for r in left:
            if p < r:
                e = new((-2, -spin(p) - spin(r)))
                e.add(1.0, opsR[("P", p, r)], I4)
                e.add(1.0, None, site_P(ints, p, r, site))
                for x in Sm:
                    dq = (-1, -spin(x) + 0)
                    dq = (-1, -(spin(p) + spin(r)) + spin(x))
                    X = _weighted([(ints.vso(p, y, r, x) - ints.vso(p, x, r, y), opsR[("d", y)])
                                   for y in Rm if (-1, -spin(y)) == dq], dq, bR)
                    e.add(1.0, X, sm[x][1])
                eo[("P", p, r)] = e
            if p <= r:
                q = r
                e = new((0, -(spin(p) - spin(q))))
                e.add(1.0, opsR[("Q", p, q)], I4)
                e.add(1.0, None, site_Q(ints, p, q, site))
                for x in Sm:
                    dq1 = (-1, -(spin(p) - spin(q)) - spin(x))
                    X1 = _weighted([(ints.vso(p, q, x, y) - ints.vso(p, y, x, q), opsR[("d", y)])
                                    for y in Rm if (-1, -spin(y)) == dq1], dq1, bR)
                    e.add(1.0, X1, sm[x][0])
                    dq2 = (1, -(spin(p) - spin(q)) + spin(x))
                    X2 = _weighted([(-(ints.vso(p, q, y, x) - ints.vso(p, x, y, q)), opsR[("d", y)].T())
                                    for y in Rm if (1, spin(y)) == dq2], dq2, bR)
                    e.add(1.0, X2, sm[x][1])
                eo[("Q", p, q)] = e
    return E, chunks, eo


def assemble_all(enl, E, chunks):
    return {k: e.assemble(E, chunks) for k, e in enl.items()}


def transform(op_enl, U, new_basis):
    """Eq. op-trans: O_new[Q'<-Q] = U_Q'^T O[Q'<-Q] U_Q over the kept sectors."""
    out = BlockOp(op_enl.dq, new_basis)
    for Q, blk in op_enl.blocks.items():
        Qo = qadd(Q, op_enl.dq)
        if Q in U and Qo in U:
            out.blocks[Q] = U[Qo].T @ blk @ U[Q]
    return out


def vacuum_left(ints):
    b = Basis([((0, 0), 1)])
    ops = {"H": BlockOp.zeros((0, 0), b)}
    for p in range(ints.n):
        ops[("RL", p)] = BlockOp.zeros((-1, -spin(p)), b)
    return b, ops


def vacuum_right(ints):
    b = Basis([((0, 0), 1)])
    ops = {"H": BlockOp.zeros((0, 0), b)}
    n = ints.n
    for p in range(n):
        ops[("RR", p)] = BlockOp.zeros((-1, -spin(p)), b)
        for r in range(p, n):
            if p < r:
                ops[("P", p, r)] = BlockOp.zeros((-2, -spin(p) - spin(r)), b)
            ops[("Q", p, r)] = BlockOp.zeros((0, -(spin(p) - spin(r))), b)
    return b, ops


__all__ = ["Integrals", "nc_terms", "count_nc_terms", "right_parity", "fock_ops_exact",
           "blocking_left", "blocking_right", "assemble_all", "transform",
           "vacuum_left", "vacuum_right", "site_basis", "spin"]
