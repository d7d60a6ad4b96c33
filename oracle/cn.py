"""U(1)xU(1) complementary/normal (CN) partition and the mixed NC/CN scheme
(oracle side).

Appendix B, Eq. h-cn gives the CN left-right decomposition in SU(2) form: the
two-index complementary operators sit on the LEFT block and the two-index
normal operators on the right. In spin orbitals (conventions of nc.py: L modes
before R modes in Jordan-Wigner order, "X (x) Y" = operator product X*Y) it
reads

  H = H_L (x) 1 + 1 (x) H_R
    + sum_{p in L} ( a+_p (x) R^R_p  -  a_p (x) (R^R_p)^T )
    + sum_{p in R} ( (R^L_p)^T (x) a_p  -  R^L_p (x) a+_p )
    + sum_{p<r in R} ( P^L_pr (x) A_pr + (P^L_pr)^T (x) A_pr^T )
    + sum_{p,q in R} Q^L_pq (x) B_pq

  P^L_pr = sum_{q,s in L} v_pqrs a_s a_q
  Q^L_pq = sum_{r,s in L} (v_pqrs - v_psrq) a+_r a_s
  A_pr = a+_p a+_r,  B_pq = a+_p a_q   (p, q, r in R)

(R^R_p, R^L_p as in nc.py; P^L and Q^L are Eq. op-def's complementary
operators summed over the left block). The two-electron part with creators
in R and annihilators in L gives the P^L (x) A terms (a+_p a+_r a_s a_q =
(a_s a_q)(a+_p a+_r) when q, s are in L and p, r in R), its conjugate the
transposed terms, and the one-creator-one-annihilator-per-side part gives
Q^L (x) B with the same coefficients as the NC B (x) Q terms.

Operator sets of a block in each form:
  left, NC  (modes [0, nL)): H, a+_p (p < nL), R^L_p (p >= nL), A_pr, B_pq (p, q, r < nL)
  left, CN:                  H, a+_p (p < nL), R^L_p (p >= nL), P^L_pr, Q^L_pq (p, q, r >= nL)
  right, NC (modes [nL, n)): H, a_p (p >= nL), R^R_p (p < nL), P_pr, Q_pq (p, q, r < nL)
  right, CN:                 H, a_p (p >= nL), R^R_p (p < nL), A_pr, B_pq (p, q, r >= nL)

Mixed NC/CN (Sec. III.A): with a cut c (spatial orbitals), a left block of k
orbitals is in NC form when k <= c and in CN form otherwise; a right block
starting at orbital k is in NC form when k <= c and in CN form otherwise. The
two-site step whose enlarged left block holds e orbitals then uses the NC
decomposition when e <= c and the CN decomposition otherwise. Blocking an
NC-form left block of c orbitals into the CN form (and a CN-form right block
starting at c+1 into the NC form) is the normal-to-complementary
transformation of the middle site: every P^L_pr / Q^L_pq of the enlarged
block is a sum of O(K^2) normal operators A / B of the old block weighted by
integrals (an O(K^4 M^2) step).

Parity status: pinned (tests/test_oracle_cn.py) - the CN decomposition
against the Fock-space Hamiltonian at every cut, every blocked operator of
the three new blocking kinds against its exact Fock-space matrix, and mixed
NC/CN sweeps at full bond dimension against FCI.
"""

import itertools

import numpy as np

from .blocks import BlockOp, enlarged_left, enlarged_right
from .nc import (EnlOp, I4, _getB, _weighted, blocking_left, site_H, site_mats,
                 site_P, site_Q, site_R, spin)


# ------------------------------------------------------------------ CN terms
def cn_terms(nL, n):
    """Canonical CN term list for L = modes [0, nL), R = modes [nL, n), in the
    format of nc.nc_terms: (left_key, left_T, right_key, right_T, coef)."""
    T = [("H", False, None, False, 1.0), (None, False, "H", False, 1.0)]
    for p in range(nL):
        T.append((("cd", p), False, ("RR", p), False, 1.0))
        T.append((("cd", p), True, ("RR", p), True, -1.0))
    for p in range(nL, n):
        T.append((("RL", p), True, ("d", p), False, 1.0))
        T.append((("RL", p), False, ("d", p), True, -1.0))
    for p in range(nL, n):
        for r in range(p + 1, n):
            T.append((("P", p, r), False, ("A", p, r), False, 1.0))
            T.append((("P", p, r), True, ("A", p, r), True, 1.0))
    for p in range(nL, n):
        for q in range(nL, n):
            if p <= q:
                T.append((("Q", p, q), False, ("B", p, q), False, 1.0))
            else:
                T.append((("Q", q, p), True, ("B", q, p), True, 1.0))
    return T


def count_cn_terms(nL, nR):
    return 2 + 2 * nL + 2 * nR + nR * (nR - 1) + nR * nR


def mixed_terms(e, K, cut):
    """Term list of the two-site step whose enlarged left block holds e
    spatial orbitals (modes [0, 2e)): NC when e <= cut, CN otherwise."""
    from .nc import nc_terms
    return nc_terms(2 * e, 2 * K) if e <= cut else cn_terms(2 * e, 2 * K)


# ---------------------------------------- complementary sums over a block
def comp_P(ints, getA, modes, p, r, bb):
    """sum_{q,s in modes} v_pqrs a_s a_q from the block's A ops:
    a_s a_q = A_qs^T (q < s), -A_sq^T (q > s), 0 (q = s)."""
    dq = (-2, -spin(p) - spin(r))
    terms = []
    for q in modes:
        for s in modes:
            x = ints.vso(p, q, r, s)
            if x == 0.0 or q == s:
                continue
            terms.append((x, getA(q, s).T()) if q < s else (-x, getA(s, q).T()))
    return _weighted(terms, dq, bb)


def comp_Q(ints, getB, modes, p, q, bb):
    """sum_{r,s in modes} (v_pqrs - v_psrq) a+_r a_s from the block's B ops."""
    dq = (0, -(spin(p) - spin(q)))
    terms = []
    for r in modes:
        for s in modes:
            x = ints.vso(p, q, r, s) - ints.vso(p, s, r, q)
            if x != 0.0:
                assert (0, spin(r) - spin(s)) == dq
                terms.append((x, getB(r, s)))
    return _weighted(terms, dq, bb)


def _pair_getter(ops, key):
    """O_pr with O_rp = -O_pr (A, P): stored for p < r."""
    def get(p, r):
        return ops[(key, p, r)] if p < r else ops[(key, r, p)].scaled(-1.0)
    return get


def _herm_getter(ops, key):
    """O_pq with O_qp = O_pq^T (B, Q): stored for p <= q."""
    def get(p, q):
        return ops[(key, p, q)] if p <= q else ops[(key, q, p)].T()
    return get


# ------------------------------------------------------------ left blocking
def blocking_left_cn(ints, bL, opsL, site, src="cn"):
    """Enlarged CN-form operators of L x site. L holds modes [0, 2*site) in CN
    form (src='cn') or in NC form (src='nc': the normal-to-complementary
    transformation). Returns (E, chunks, enl_ops) keyed like a CN left block
    of modes [0, 2*site+2)."""
    n = ints.n
    Lm = list(range(0, 2 * site))
    Sm = [2 * site, 2 * site + 1]
    sm = site_mats(site)
    E, chunks = enlarged_left(bL)
    eo = {}

    def new(dq):
        return EnlOp("L", dq, bL)

    if src == "nc":
        getA, getB = _pair_getter(opsL, "A"), _herm_getter(opsL, "B")
        PL = lambda p, r: comp_P(ints, getA, Lm, p, r, bL)
        QL = lambda p, q: comp_Q(ints, getB, Lm, p, q, bL)
    else:
        PL, QL = _pair_getter(opsL, "P"), _herm_getter(opsL, "Q")

    for p in Lm:
        eo[("cd", p)] = new((1, spin(p))).add(1.0, opsL[("cd", p)], I4)
    for p in Sm:
        eo[("cd", p)] = new((1, spin(p))).add(1.0, None, sm[p][0])

    # H of L x s at the cut (L | s)
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
    if src == "nc":  # NC form: normal pairs of L with the site's complementary parts
        getA = _pair_getter(opsL, "A")
        for p in Lm:
            for r in Lm:
                if p < r:
                    Ps = site_P(ints, p, r, site)
                    e.add(1.0, getA(p, r), Ps)
                    e.add(1.0, getA(p, r).T(), Ps.T)
        for p in Lm:
            for q in Lm:
                e.add(1.0, _getB(opsL, p, q), site_Q(ints, p, q, site))
    else:  # CN form: complementary pairs of L with the site's normal pairs
        p, r = Sm
        A = sm[p][0] @ sm[r][0]
        e.add(1.0, PL(p, r), A)
        e.add(1.0, PL(p, r).T(), A.T)
        for p in Sm:
            for q in Sm:
                e.add(1.0, QL(p, q), sm[p][0] @ sm[q][1])
    eo["H"] = e

    right = list(range(2 * site + 2, n))
    for p in right:  # R^L_p, no one-body part
        e = new((-1, -spin(p)))
        e.add(1.0, opsL[("RL", p)], I4)
        e.add(1.0, None, site_R(ints, p, site, one_body=False))
        for x in Sm:  # r, s in L, q = x on the site: Q^L_px (x) a_x
            e.add(1.0, QL(p, x), sm[x][1])
        for r in Sm:  # q, s in L, r on the site: P^L_pr (x) a+_r
            e.add(1.0, PL(p, r), sm[r][0])
        for s in Lm:  # q, r on the site; s in L: -a_s (x) a+_r a_q
            m = np.zeros((4, 4))
            for q in Sm:
                for r in Sm:
                    m += ints.vso(p, q, r, s) * sm[r][0] @ sm[q][1]
            if np.any(m):
                e.add(-1.0, opsL[("cd", s)].T(), m)
        for r in Lm:  # q, s on the site; r in L: a+_r (x) a_s a_q
            m = np.zeros((4, 4))
            for q in Sm:
                for s in Sm:
                    m += ints.vso(p, q, r, s) * sm[s][1] @ sm[q][1]
            if np.any(m):
                e.add(1.0, opsL[("cd", r)], m)
        for q in Lm:  # r, s on the site; q in L: a_q (x) a+_r a_s
            m = np.zeros((4, 4))
            for r in Sm:
                for s in Sm:
                    m += ints.vso(p, q, r, s) * sm[r][0] @ sm[s][1]
            if np.any(m):
                e.add(1.0, opsL[("cd", q)].T(), m)
        eo[("RL", p)] = e

    for p in right:
        for r in right:
            if p < r:  # P^L_pr = sum_{q,s in L+s} v_pqrs a_s a_q
                e = new((-2, -spin(p) - spin(r)))
                e.add(1.0, PL(p, r), I4)
                e.add(1.0, None, site_P(ints, p, r, site))
                for x in Sm:  # one of q, s on the site, the other (y) in L
                    dq = (-1, -(spin(p) + spin(r)) + spin(x))
                    X = _weighted([(ints.vso(p, x, r, y) - ints.vso(p, y, r, x), opsL[("cd", y)].T())
                                   for y in Lm if (-1, -spin(y)) == dq], dq, bL)
                    e.add(1.0, X, sm[x][1])
                eo[("P", p, r)] = e
            if p <= r:  # Q^L_pq = sum_{r',s in L+s} (v_pqr's - v_psr'q) a+_r' a_s
                q = r
                e = new((0, -(spin(p) - spin(q))))
                e.add(1.0, QL(p, q), I4)
                e.add(1.0, None, site_Q(ints, p, q, site))
                for x in Sm:
                    # creator y in L, annihilator x on the site: a+_y (x) a_x
                    dq1 = (1, -(spin(p) - spin(q)) + spin(x))
                    X1 = _weighted([(ints.vso(p, q, y, x) - ints.vso(p, x, y, q), opsL[("cd", y)])
                                    for y in Lm if (1, spin(y)) == dq1], dq1, bL)
                    e.add(1.0, X1, sm[x][1])
                    # creator x on the site, annihilator y in L: -a_y (x) a+_x
                    dq2 = (-1, -(spin(p) - spin(q)) - spin(x))
                    X2 = _weighted([(-(ints.vso(p, q, x, y) - ints.vso(p, y, x, q)), opsL[("cd", y)].T())
                                    for y in Lm if (-1, -spin(y)) == dq2], dq2, bL)
                    e.add(1.0, X2, sm[x][0])
                eo[("Q", p, q)] = e
    return E, chunks, eo


def blocking_left_mixed(ints, bL, opsL, site, cut):
    """Left blocking under the mixed scheme: the enlarged block (site+1
    orbitals) is NC when site+1 <= cut, else CN (from an NC block at
    site == cut: the transformation)."""
    if site + 1 <= cut:
        return blocking_left(ints, bL, opsL, site)
    return blocking_left_cn(ints, bL, opsL, site, "nc" if site <= cut else "cn")


# ----------------------------------------------------------- right blocking
def blocking_right_cn(ints, bR, opsR, site, dst="cn"):
    """Enlarged operators of site x R with R (modes [2*site+2, n)) in CN form.
    dst='cn': the enlarged block in CN form (A, B over its modes); dst='nc':
    in NC form (P, Q over the modes left of it: the transformation).
    Returns (E, chunks, enl_ops)."""
    n = ints.n
    Rm = list(range(2 * site + 2, n))
    Sm = [2 * site, 2 * site + 1]
    sm = site_mats(site)
    E, chunks = enlarged_right(bR)
    eo = {}
    getA, getB = _pair_getter(opsR, "A"), _herm_getter(opsR, "B")
    PR = lambda p, r: comp_P(ints, getA, Rm, p, r, bR)
    QR = lambda p, q: comp_Q(ints, getB, Rm, p, q, bR)

    def new(dq):
        return EnlOp("R", dq, bR)

    for p in Sm:
        eo[("d", p)] = new((-1, -spin(p))).add(1.0, None, sm[p][1])
    for p in Rm:
        eo[("d", p)] = new((-1, -spin(p))).add(1.0, opsR[("d", p)], I4)

    # H of s x R at the cut (s | R), CN form: complementary parts on the site
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
    for p in Rm:
        for r in Rm:
            if p < r:
                Ps = site_P(ints, p, r, site)
                e.add(1.0, getA(p, r), Ps)
                e.add(1.0, getA(p, r).T(), Ps.T)
    for p in Rm:
        for q in Rm:
            e.add(1.0, getB(p, q), site_Q(ints, p, q, site))
    eo["H"] = e

    left = list(range(0, 2 * site))
    for p in left:  # R^R_p with its one-body part
        e = new((-1, -spin(p)))
        e.add(1.0, opsR[("RR", p)], I4)
        e.add(1.0, None, site_R(ints, p, site, one_body=True))
        for x in Sm:
            e.add(1.0, QR(p, x), sm[x][1])  # q = x on the site: a_x (x) Q^R_px
            e.add(1.0, PR(p, x), sm[x][0])  # r = x on the site: a+_x (x) P^R_px
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

    newm = Sm + Rm
    if dst == "cn":
        for p in newm:
            for r in newm:
                if p < r:  # A_pr
                    e = new((2, spin(p) + spin(r)))
                    if p in Rm:
                        e.add(1.0, opsR[("A", p, r)], I4)
                    elif r in Rm:  # a+_p (site) a+_r (block)
                        e.add(1.0, opsR[("d", r)].T(), sm[p][0])
                    else:
                        e.add(1.0, None, sm[p][0] @ sm[r][0])
                    eo[("A", p, r)] = e
                if p <= r:  # B_pq
                    q = r
                    e = new((0, spin(p) - spin(q)))
                    if p in Rm:
                        e.add(1.0, opsR[("B", p, q)], I4)
                    elif q in Rm:  # a+_p (site) a_q (block)
                        e.add(1.0, opsR[("d", q)], sm[p][0])
                    else:
                        e.add(1.0, None, sm[p][0] @ sm[q][1])
                    eo[("B", p, q)] = e
        return E, chunks, eo

    for p in left:
        for r in left:
            if p < r:  # P_pr = sum_{q,s in s+R} v_pqrs a_s a_q
                e = new((-2, -spin(p) - spin(r)))
                e.add(1.0, PR(p, r), I4)
                e.add(1.0, None, site_P(ints, p, r, site))
                for x in Sm:
                    dq = (-1, -(spin(p) + spin(r)) + spin(x))
                    X = _weighted([(ints.vso(p, y, r, x) - ints.vso(p, x, r, y), opsR[("d", y)])
                                   for y in Rm if (-1, -spin(y)) == dq], dq, bR)
                    e.add(1.0, X, sm[x][1])
                eo[("P", p, r)] = e
            if p <= r:  # Q_pq = sum_{r',s in s+R} (v_pqr's - v_psr'q) a+_r' a_s
                q = r
                e = new((0, -(spin(p) - spin(q))))
                e.add(1.0, QR(p, q), I4)
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


def blocking_right_mixed(ints, bR, opsR, site, cut):
    """Right blocking under the mixed scheme: the enlarged block starts at
    orbital `site`; NC form when site <= cut, else CN. R starts at site+1."""
    from .nc import blocking_right
    if site + 1 <= cut:
        return blocking_right(ints, bR, opsR, site)
    return blocking_right_cn(ints, bR, opsR, site, "nc" if site <= cut else "cn")


def vacuum_right_cn(ints):
    """Empty right block in CN form: H and R^R_p for every mode, all zero."""
    from .blocks import Basis
    b = Basis([((0, 0), 1)])
    ops = {"H": BlockOp.zeros((0, 0), b)}
    for p in range(ints.n):
        ops[("RR", p)] = BlockOp.zeros((-1, -spin(p)), b)
    return b, ops


__all__ = ["cn_terms", "count_cn_terms", "mixed_terms", "comp_P", "comp_Q", "blocking_left_cn",
           "blocking_left_mixed", "blocking_right_cn", "blocking_right_mixed", "vacuum_right_cn"]
