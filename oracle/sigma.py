"""H_eff . psi as a sum over NC terms of block-sparse products (oracle side).

Sec. II.D-E: the Davidson matrix-vector product is a sum over left-right
operator pairs (Eq. hpsi-thread and the reduction that follows it); each
term is a block-sparse product that splits into dense products over
symmetry sectors. With psi stored as a matrix psi[l, r] over the product
basis of the two (enlarged) blocks, one term c * X (x) Y contributes

    sigma[q_L + dX, q_R + dY] += c * (-1)^(|Y| N(q_L)) X[q_L+dX <- q_L] psi[q_L, q_R] Y[q_R+dY <- q_R]^T

(sign from moving Y past the left block's creation operators). psi is
block-diagonal over (q_L, Q_tot - q_L): blocks ordered by q_L ascending, each
block row-major m_L x m_R.

This file also builds the synthetic middle-bond operator layout (random
blocks drawn by the counter-based generator, see splitmix.py): the stored
operators of an NC left block (H, a+_p, R^L_p, A_pr, B_pq) and of an NC
right block (H, a_p, R^R_p, P_pr, Q_pq) over given sector lists.

Parity status: pinned. sigma_blocks with exact Fock-space operators equals
H . psi (tests/test_oracle_nc.py); the synthetic operator set gives a
symmetric H_eff and the published term count (tests/test_oracle_sigma.py).
"""

import numpy as np

from . import splitmix
from .blocks import Basis, BlockOp, qadd, qsub
from .nc import nc_terms, right_parity, spin


# ------------------------------------------------------------- psi layout
def psi_layout(bL, bR, Qtot):
    """List of (q_L, q_R, m_L, m_R, offset) for psi blocks, q_L ascending."""
    out, off = [], 0
    for qL in bL.qs:
        qR = qsub(Qtot, qL)
        if bR.has(qR):
            mL, mR = bL.dim(qL), bR.dim(qR)
            out.append((qL, qR, mL, mR, off))
            off += mL * mR
    return out, off


def psi_to_blocks(vec, layout):
    return {qL: vec[off:off + mL * mR].reshape(mL, mR) for qL, qR, mL, mR, off in layout}


def blocks_to_psi(blocks, layout, size):
    v = np.zeros(size)
    for qL, qR, mL, mR, off in layout:
        if qL in blocks:
            v[off:off + mL * mR] = blocks[qL].ravel()
    return v


def _used(op, trans):
    return op.T() if trans else op


def sigma_blocks(psi_vec, layout, terms, opsL, opsR, term_range=None):
    """sigma = H_eff psi (plain per-term, per-block numpy loop)."""
    psi = psi_to_blocks(psi_vec, layout)
    sig = {qL: np.zeros((mL, mR)) for qL, qR, mL, mR, off in layout}
    qR_of = {qL: qR for qL, qR, mL, mR, off in layout}
    lo, hi = (0, len(terms)) if term_range is None else term_range
    for kl, tl, kr, tr, c in terms[lo:hi]:
        X = None if kl is None else _used(opsL[kl], tl)
        Y = None if kr is None else _used(opsR[kr], tr)
        par = right_parity(kr)
        for qL, blk in psi.items():
            qR = qR_of[qL]
            qLo = qL if X is None else qadd(qL, X.dq)
            qRo = qR if Y is None else qadd(qR, Y.dq)
            if qLo not in sig or qR_of[qLo] != qRo:
                continue
            if X is not None and qL not in X.blocks:
                continue
            if Y is not None and qR not in Y.blocks:
                continue
            t = blk if X is None else X.blocks[qL] @ blk
            t = t if Y is None else t @ Y.blocks[qR].T
            sign = -1.0 if (par and qL[0] % 2) else 1.0
            sig[qLo] += (c * sign) * t
    return blocks_to_psi(sig, layout, sum(m * n for _, _, m, n, _ in layout))


# ------------------------------------------------- sub-Hamiltonian split
def proc_one(i, P):
    """Eq. proc-def, one index (0-based ranks and indices): i mod P."""
    return i % P


def proc_two(i, j, P):
    """Eq. proc-def, two indices: the rank of the pair depends only on the
    unordered pair {i, j}; with i <= j (1-based) it is (j-1)j/2 + i mod P,
    i.e. j(j+1)/2 + i mod P for 0-based i <= j."""
    lo, hi = min(i, j), max(i, j)
    return (hi * (hi + 1) // 2 + lo) % P


def nc_term_rank(term, P):
    """Rank of one NC term under the NC partition of Eq. proc-def-nc, in
    spin-orbital indices: a term's rank follows the left-block indices of its
    left operator (a+_p, R^L_p: one index; A_pr, B_pq: the pair); the terms
    H_L x 1 and 1 x H_R, which carry no pair, go to rank 0."""
    kl = term[0]
    if kl is None or kl == "H":
        return 0
    if kl[0] in ("cd", "RL"):
        return proc_one(kl[1], P)
    return proc_two(kl[1], kl[2], P)


def sigma_part(psi_vec, layout, terms, opsL, opsR, rank, P):
    """sigma of sub-Hamiltonian `rank` of P (Sec. II.B, Eq. sum-h): the terms
    that nc_term_rank assigns to it."""
    mine = [t for t in terms if nc_term_rank(t, P) == rank]
    return sigma_blocks(psi_vec, layout, mine, opsL, opsR)


def heff_diagonal(layout, terms, opsL, opsR):
    """Diagonal of H_eff (terms whose left and right shifts are both zero)."""
    size = sum(m * n for _, _, m, n, _ in layout)
    d = np.zeros(size)
    for kl, tl, kr, tr, c in terms:
        X = None if kl is None else opsL[kl]
        Y = None if kr is None else opsR[kr]
        if (X is not None and X.dq != (0, 0)) or (Y is not None and Y.dq != (0, 0)):
            continue
        for qL, qR, mL, mR, off in layout:
            dl = np.ones(mL) if X is None else (np.diag(X.blocks[qL]) if qL in X.blocks else None)
            dr = np.ones(mR) if Y is None else (np.diag(Y.blocks[qR]) if qR in Y.blocks else None)
            if dl is None or dr is None:
                continue
            d[off:off + mL * mR] += c * np.outer(dl, dr).ravel()
    return d


def heff_dense(layout, terms, opsL, opsR):
    """Explicit H_eff matrix (columns = sigma of unit vectors); tiny cases only."""
    size = sum(m * n for _, _, m, n, _ in layout)
    H = np.zeros((size, size))
    for j in range(size):
        e = np.zeros(size)
        e[j] = 1.0
        H[:, j] = sigma_blocks(e, layout, terms, opsL, opsR)
    return H


# ---------------------------------------------------- synthetic operator set
def synthetic_op_specs(nL_modes, n_modes):
    """Canonical stored-operator list: [(side, key, dq, symmetric)], left side
    first. Left: H, a+_p (p in L), R^L_p (p in R), A_pr (p<r in L), B_pq (p<=q
    in L). Right: H, a_p (p in R), R^R_p (p in L), P_pr (p<r in L), Q_pq (p<=q in L).
    H, B_pp and Q_pp are symmetric (only their upper triangle is drawn)."""
    L = range(nL_modes)
    R = range(nL_modes, n_modes)
    out = [("L", "H", (0, 0), True)]
    out += [("L", ("cd", p), (1, spin(p)), False) for p in L]
    out += [("L", ("RL", p), (-1, -spin(p)), False) for p in R]
    out += [("L", ("A", p, r), (2, spin(p) + spin(r)), False) for p in L for r in L if p < r]
    out += [("L", ("B", p, q), (0, spin(p) - spin(q)), p == q) for p in L for q in L if p <= q]
    out += [("R", "H", (0, 0), True)]
    out += [("R", ("d", p), (-1, -spin(p)), False) for p in R]
    out += [("R", ("RR", p), (-1, -spin(p)), False) for p in L]
    out += [("R", ("P", p, r), (-2, -spin(p) - spin(r)), False) for p in L for r in L if p < r]
    out += [("R", ("Q", p, q), (0, -(spin(p) - spin(q))), p == q) for p in L for q in L if p <= q]
    return out


def synthetic_block_table(specs, bL, bR):
    """For every stored op, its blocks [(q_in, q_out, rows, cols, flat_offset)]
    in canonical order (ops in spec order, blocks by ascending q_in, row-major)."""
    dims = {"L": dict(zip(bL.qs, bL.dims)), "R": dict(zip(bR.qs, bR.dims))}
    qs = {"L": bL.qs, "R": bR.qs}
    table, off = [], 0
    for side, key, dq, sym in specs:
        d = dims[side]
        blks = []
        for q in qs[side]:
            qo = (q[0] + dq[0], q[1] + dq[1])
            r = d.get(qo)
            if r is not None:
                c = d[q]
                blks.append((q, qo, r, c, off))
                off += r * c
        table.append(blks)
    return table, off


def _block_values(key, off, r, c, sym):
    idx = np.arange(r * c, dtype=np.int64).reshape(r, c)
    if sym:
        i, j = np.indices((r, c))
        idx = np.where(i <= j, i * c + j, j * c + i)
    return splitmix.normal(key, (off + idx).astype(np.uint64))


def synthetic_ops(left_secs, right_secs, nL_modes, n_modes, seed, only=None):
    """Build the synthetic operator dicts (opsL, opsR) with N(0,1) entries.

    left_secs/right_secs: [(N, 2Sz, dim)]. Element (i, j) of a block with flat
    canonical offset `off` takes counter off + i*cols + j (for symmetric
    operators, the counter of (min, max)). only: optional set of (side, key)
    to build (others skipped; offsets stay canonical)."""
    bL = Basis([((n, s), d) for n, s, d in left_secs])
    bR = Basis([((n, s), d) for n, s, d in right_secs])
    specs = synthetic_op_specs(nL_modes, n_modes)
    table, total = synthetic_block_table(specs, bL, bR)
    key = splitmix.stream_key(seed, splitmix.KEY_OPS)
    opsL, opsR = {}, {}
    for (side, k, dq, sym), blks in zip(specs, table):
        if only is not None and (side, k) not in only:
            continue
        b = bL if side == "L" else bR
        op = BlockOp(dq, b)
        for q, qo, r, c, off in blks:
            op.blocks[q] = _block_values(key, off, r, c, sym)
        (opsL if side == "L" else opsR)[k] = op
    return bL, bR, opsL, opsR, total


def sigma_flops(layout, terms, dqL, dqR, bL, bR):
    """Algorithmic FLOPs of one sigma (2 per multiply-add): per term and psi
    block, the cheaper of the two contraction orders (X psi) Y^T and X (psi Y^T);
    identity factors cost nothing. dqL/dqR: key -> shift of the stored op."""
    total = 0
    blk = {qL: (qR, mL, mR) for qL, qR, mL, mR, off in layout}
    for kl, tl, kr, tr, c in terms:
        dx = (0, 0) if kl is None else (dqL[kl] if not tl else (-dqL[kl][0], -dqL[kl][1]))
        dy = (0, 0) if kr is None else (dqR[kr] if not tr else (-dqR[kr][0], -dqR[kr][1]))
        for qL, (qR, m, n) in blk.items():
            qLo, qRo = qadd(qL, dx), qadd(qR, dy)
            if qLo not in blk or blk[qLo][0] != qRo:
                continue
            mo, no = blk[qLo][1], blk[qLo][2]
            if kl is None:
                total += 2 * m * n * no
            elif kr is None:
                total += 2 * mo * m * n
            else:
                total += min(2 * mo * m * n + 2 * mo * n * no, 2 * m * n * no + 2 * mo * m * no)
    return total


def _block_rows(key, off, r, c, sym, rows, trans):
    """Rows `rows` of a stored block (r x c, canonical offset off), or of its
    transpose when trans, drawn element by element from their counters."""
    rows = np.asarray(rows, dtype=np.int64)
    if not trans:
        i = rows[:, None]
        j = np.arange(c, dtype=np.int64)[None, :]
    else:  # rows of S^T = columns of S
        i = np.arange(r, dtype=np.int64)[None, :]
        j = rows[:, None]
    if sym:
        i, j = np.minimum(i, j), np.maximum(i, j)
    return splitmix.normal(key, (off + i * c + j).astype(np.uint64))


def synthetic_sigma_sampled(left_secs, right_secs, nL_modes, n_modes, seed, Qtot, psi_vec,
                            samples):
    """Selected entries of sigma for the synthetic operator set: samples is
    [(q_L, rows, cols)] and the result {q_L: sigma[q_L][ix_(rows, cols)]}.
    Only the operator rows those entries need are drawn, so this runs at the
    full benchmark size."""
    bL = Basis([((n, s), d) for n, s, d in left_secs])
    bR = Basis([((n, s), d) for n, s, d in right_secs])
    specs = synthetic_op_specs(nL_modes, n_modes)
    table, _ = synthetic_block_table(specs, bL, bR)
    key = splitmix.stream_key(seed, splitmix.KEY_OPS)
    index = {(side, k): (dq, sym) for (side, k, dq, sym) in specs}
    by_in = {(side, k): {q: (qo, r, c, off) for q, qo, r, c, off in blks}
             for (side, k, dq, sym), blks in zip(specs, table)}
    by_out = {(side, k): {qo: (q, r, c, off) for q, qo, r, c, off in blks}
              for (side, k, dq, sym), blks in zip(specs, table)}
    layout, size = psi_layout(bL, bR, Qtot)
    psi = psi_to_blocks(psi_vec, layout)
    qR_of = {qL: qR for qL, qR, mL, mR, off in layout}
    want = {tuple(q): (np.asarray(r), np.asarray(c)) for q, r, c in samples}
    out = {q: np.zeros((len(r), len(c))) for q, (r, c) in want.items()}

    def used_rows(side, k, trans, qin, rows):
        sym = index[(side, k)][1]
        hit = (by_out if trans else by_in)[(side, k)].get(qin)
        if hit is None:
            return None, None
        qo, r, c, off = hit
        return qo, _block_rows(key, off, r, c, sym, rows, trans)

    for kl, tl, kr, tr, c in nc_terms(nL_modes, n_modes):
        par = right_parity(kr)
        if kl is None:
            dxl = (0, 0)
        else:
            dq = index[("L", kl)][0]
            dxl = (-dq[0], -dq[1]) if tl else dq
        for qLo, (rows, cols) in want.items():
            qL = qsub(qLo, dxl)
            if qL not in psi:
                continue
            blk = psi[qL]
            qR = qR_of[qL]
            if kl is None:
                X = blk[rows, :]
            else:
                q2, X = used_rows("L", kl, tl, qL, rows)
                if q2 is None:
                    continue
            if kr is None:
                qRo, Y = qR, None
            else:
                qRo, Y = used_rows("R", kr, tr, qR, cols)
                if qRo is None:
                    continue
            if qR_of.get(qLo) != qRo:
                continue
            t = X if kl is None else X @ blk
            t = t[:, cols] if Y is None else t @ Y.T
            sign = -1.0 if (par and qL[0] % 2) else 1.0
            out[qLo] += (c * sign) * t
    return out
