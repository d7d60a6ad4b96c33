"""Quantum-number bases and block-sparse operators (oracle side).

A Basis is an ascending list of sectors q = (N, 2Sz) with dimensions. A
BlockOp with shift dq maps sector q of its input basis to sector q + dq of
its output basis; it stores one dense FP64 block per input sector for which
both sectors exist (Sec. II.E: block-sparse matrices over symmetry sectors).
Its fermion parity is dN mod 2.

Enlarged bases (Eq. blocked-ops): the product of a block basis and one site
basis. An enlarged sector Q is a concatenation of chunks, one per block sector
q_b with q_b + q_site = Q, in ascending q_b; the block state index runs
inside a chunk. For a site on the right of the block (left enlarged block
L x s) and on the left of it (right enlarged block s x R) the chunk order is
the same rule.

Parity status: pinned through the tests of nc.py / dmrg.py, which compare
block-sparse results with dense Fock-space matrices.
"""

import numpy as np


def qadd(a, b):
    return (a[0] + b[0], a[1] + b[1])


def qsub(a, b):
    return (a[0] - b[0], a[1] - b[1])


class Basis:
    def __init__(self, sectors):
        """sectors: iterable of ((N, 2Sz), dim); zero dims are dropped."""
        secs = sorted((tuple(q), int(d)) for q, d in sectors if int(d) > 0)
        self.qs = [q for q, _ in secs]
        self.dims = [d for _, d in secs]
        self.index = {q: k for k, q in enumerate(self.qs)}
        self.offsets = np.concatenate([[0], np.cumsum(self.dims)]).astype(np.int64)
        self.total = int(self.offsets[-1])

    def dim(self, q):
        k = self.index.get(q)
        return 0 if k is None else self.dims[k]

    def has(self, q):
        return q in self.index

    def __repr__(self):
        return f"Basis({list(zip(self.qs, self.dims))})"


class BlockOp:
    """Block-sparse operator: blocks[q_in] has shape (dim_out(q_in+dq), dim_in(q_in))."""

    def __init__(self, dq, bin_, bout=None, blocks=None):
        self.dq = tuple(dq)
        self.bin = bin_
        self.bout = bin_ if bout is None else bout
        self.blocks = {} if blocks is None else blocks

    @property
    def parity(self):
        return self.dq[0] % 2

    @staticmethod
    def zeros(dq, bin_, bout=None):
        op = BlockOp(dq, bin_, bout)
        for q in op.bin.qs:
            qo = qadd(q, op.dq)
            if op.bout.has(qo):
                op.blocks[q] = np.zeros((op.bout.dim(qo), op.bin.dim(q)))
        return op

    @staticmethod
    def identity(b):
        return BlockOp((0, 0), b, b, {q: np.eye(b.dim(q)) for q in b.qs})

    def T(self):
        """Transpose (= Hermitian conjugate for real matrices)."""
        out = BlockOp((-self.dq[0], -self.dq[1]), self.bout, self.bin)
        for q, blk in self.blocks.items():
            out.blocks[qadd(q, self.dq)] = blk.T.copy()
        return out

    def scaled(self, c):
        return BlockOp(self.dq, self.bin, self.bout, {q: c * b for q, b in self.blocks.items()})

    def axpy(self, c, other):
        """self += c * other (same shift and bases)."""
        assert other.dq == self.dq
        for q, blk in other.blocks.items():
            if q in self.blocks:
                self.blocks[q] += c * blk
            else:
                self.blocks[q] = c * blk.copy()
        return self

    def to_dense(self):
        D = np.zeros((self.bout.total, self.bin.total))
        for q, blk in self.blocks.items():
            qo = qadd(q, self.dq)
            i0 = self.bout.offsets[self.bout.index[qo]]
            j0 = self.bin.offsets[self.bin.index[q]]
            D[i0:i0 + blk.shape[0], j0:j0 + blk.shape[1]] = blk
        return D

    @staticmethod
    def from_dense(D, dq, bin_, bout=None):
        op = BlockOp(dq, bin_, bout)
        for q in op.bin.qs:
            qo = qadd(q, op.dq)
            if op.bout.has(qo):
                i0 = op.bout.offsets[op.bout.index[qo]]
                j0 = op.bin.offsets[op.bin.index[q]]
                op.blocks[q] = D[i0:i0 + op.bout.dim(qo), j0:j0 + op.bin.dim(q)].copy()
        return op

    def nnz_elements(self):
        return sum(b.size for b in self.blocks.values())


# ----------------------------------------------------------------- site basis
# One spatial orbital = two spin orbitals (alpha first in Jordan-Wigner order).
# Local states as integers with bit0 = alpha, bit1 = beta:
#   0 = |0>, 1 = |a> = a+_a|0>, 2 = |b> = a+_b|0>, 3 = |ab> = a+_a a+_b |0>.
SITE_Q = {0: (0, 0), 1: (1, 1), 2: (1, -1), 3: (2, 0)}
SITE_N = {0: 0, 1: 1, 2: 1, 3: 2}


def site_basis():
    return Basis([(SITE_Q[n], 1) for n in range(4)])


def site_cre(sigma):
    """4x4 matrix of a+_sigma on one spatial orbital (local JW order alpha, beta)."""
    m = np.zeros((4, 4))
    for s in range(4):
        if not (s >> sigma) & 1:
            sign = -1.0 if (sigma == 1 and (s & 1)) else 1.0
            m[s | (1 << sigma), s] = sign
    return m


def enlarged_left(bL):
    """Basis of L x s and its chunk table {Q: [(q_L, n, offset_in_Q)]}."""
    secs, chunks = {}, {}
    for q in bL.qs:  # ascending q_L
        for n in range(4):
            Q = qadd(q, SITE_Q[n])
            off = secs.get(Q, 0)
            chunks.setdefault(Q, []).append((q, n, off))
            secs[Q] = off + bL.dim(q)
    return Basis(list(secs.items())), chunks


def enlarged_right(bR):
    """Basis of s x R and its chunk table {Q: [(q_R, n, offset_in_Q)]} (ascending q_R)."""
    secs, chunks = {}, {}
    for q in bR.qs:
        for n in range(4):
            Q = qadd(q, SITE_Q[n])
            off = secs.get(Q, 0)
            chunks.setdefault(Q, []).append((q, n, off))
            secs[Q] = off + bR.dim(q)
    return Basis(list(secs.items())), chunks
