"""Plain two-site ab initio DMRG with the U(1)xU(1) NC partition (oracle side).

Follows Appendix A: for each sweep iteration at sites (i, i+1),
  (i)  blocking: enlarged blocks L_i x s_i and s_{i+1} x R_{i+2}
       (Eq. blocked-ops; formulas in nc.blocking_left / blocking_right and,
       for the CN form, cn.blocking_left_cn / blocking_right_cn);
  (ii) solving: lowest eigenpair of H_eff (Eq. eff-eigsh) by Davidson, with
       the NC sigma of sigma.sigma_blocks;
  (iii) decimation by SVD of psi per sector block and truncation to M, then
       transformation of the growing block's operators (Eq. op-trans).
Forward sweeps move the canonical centre right (keep U), backward sweeps
move it left (keep V^T).

Fixed readings of points the paper leaves open:
  * Initial MPS: right blocks R_j (spatial orbitals j..K-1) are built right to
    left; the kept sectors of s_j x R_{j+1} are those the left part
    (2j spin orbitals) can complement to the target (N, 2Sz); if their total
    dimension exceeds M_init, sector dims are the largest-remainder rounding
    of M_init * d_Q / D (ties by ascending Q). The basis of sector Q is the
    orthonormalised column space of a random d_Q x m_Q matrix whose entries
    are SplitMix64 normals (key = seed ^ KEY_MPS, counter = running flat
    offset over j descending, Q ascending, row-major).
  * Truncation: all singular values of all psi blocks sorted by
    (s descending, q_L ascending, index ascending); the first
    min(M, count) are kept, zero singular values included.
  * Davidson guess at each step: the previous step's wavefunction carried to
    the new bond (the sweep moves one site; the previous psi is projected on
    the block just kept and the block it leaves is expanded through the
    stored basis of the next block: predict()); at the turn of a sweep the
    bond and blocks are unchanged and the previous psi is the guess. The
    first step after build_blocks uses SplitMix64 normals (key = seed ^
    KEY_GUESS, counter = step_id * 2^32 + element index, step_id =
    sweep * K + i).
  * Sweep energy: the lowest Davidson eigenvalue of the sweep.
  * Mixed NC/CN (Sec. III.A, cn.py): with cut c, blocks of at most c left
    orbitals / starting at orbital c or before are in NC form, the others in
    CN form; the step whose enlarged left block holds e orbitals uses the NC
    terms when e <= c, the CN terms otherwise. cut=None is NC everywhere.

Parity status: pinned (tests/test_oracle_dmrg.py): at full bond dimension
every sweep energy equals the FCI energy; blocked operators equal their
Fock-space matrices; renormalized bases are orthonormal.
"""

import numpy as np

from . import splitmix
from .blocks import SITE_Q, Basis, BlockOp, enlarged_left, enlarged_right, qadd, qsub
from .davidson import davidson
from .cn import blocking_left_mixed, blocking_right_mixed, mixed_terms, vacuum_right_cn
from .nc import Integrals, assemble_all, transform, vacuum_left, vacuum_right
from .sigma import blocks_to_psi, heff_diagonal, psi_layout, psi_to_blocks, sigma_blocks


def can_hold(n_modes, q):
    N, s = q
    return 0 <= N <= n_modes and (s - N) % 2 == 0 and abs(s) <= min(N, n_modes - N)


def largest_remainder(total, weights):
    w = np.asarray(weights, dtype=np.float64)
    exact = total * w / w.sum()
    base = np.floor(exact).astype(np.int64)
    short = int(total - base.sum())
    order = sorted(range(len(w)), key=lambda a: (-(exact[a] - base[a]), a))
    for a in order[:short]:
        base[a] += 1
    return base


def fix_sign(U):
    """Columns with the sign that makes each column's entry of largest
    magnitude positive (the first such entry on ties): singular vectors have
    an arbitrary sign, and this fixes the gauge of the kept states."""
    U = np.array(U, dtype=np.float64)
    for j in range(U.shape[1]):
        i = int(np.argmax(np.abs(U[:, j])))
        if U[i, j] < 0.0:
            U[:, j] = -U[:, j]
    return U


def orthonormal_columns(G):
    """Orthonormal basis of the columns of G in Gram-Schmidt orientation:
    the unique thin QR with a positive diagonal of R, so the basis (and every
    block built on it) is a function of G alone, not of the QR routine."""
    Q, R = np.linalg.qr(G)
    sgn = np.where(np.diag(R) < 0.0, -1.0, 1.0)
    return Q * sgn


class PlainDMRG:
    def __init__(self, t, v, N, two_sz, seed=0, dav_tol=1e-10, dav_max_space=24,
                 dav_max_iter=200, noise=0.0, keep_one_per_q=False, cut=None):
        self.ints = Integrals(t, v)
        self.K = self.ints.K
        self.cut = self.K if cut is None else int(cut)
        self.Q = (N, two_sz)
        self.seed = seed
        self.dav = dict(tol=dav_tol, max_space=dav_max_space, max_iter=dav_max_iter)
        self.noise = float(noise)
        self.keep_one_per_q = bool(keep_one_per_q)
        self.L = {}
        self.R = {}
        self.UL = {}  # i -> {sector of L[i-1] x site: kept columns}, for inspection
        self.UR = {}  # j -> {sector of site x R[j+1]: kept columns}
        self.log = []
        self.prev = None  # (i, forward, psi, layout) of the last step

    # ------------------------------------------------------ initial blocks
    def build_blocks(self, M_init):
        K = self.K
        self.R[K] = vacuum_right(self.ints) if K <= self.cut else vacuum_right_cn(self.ints)
        key = splitmix.stream_key(self.seed, splitmix.KEY_MPS)
        off = 0
        for j in range(K - 1, 0, -1):
            bR, opsR = self.R[j + 1]
            E, chunks, enl = blocking_right_mixed(self.ints, bR, opsR, j, self.cut)
            comp = [(Q, E.dim(Q)) for Q in E.qs if can_hold(2 * j, qsub(self.Q, Q))]
            D = sum(d for _, d in comp)
            dims = [d for _, d in comp] if D <= M_init else list(largest_remainder(M_init, [d for _, d in comp]))
            U, secs = {}, []
            for (Q, d), m in zip(comp, dims):
                if m <= 0:
                    continue
                g = splitmix.normal(key, np.arange(off, off + d * m, dtype=np.uint64)).reshape(d, m)
                off += d * m
                U[Q] = orthonormal_columns(g)
                secs.append((Q, m))
            nb = Basis(secs)
            ops = {k: transform(e.assemble(E, chunks), U, nb) for k, e in enl.items()}
            self.R[j] = (nb, ops)
            self.UR[j] = U
        self.L[0] = vacuum_left(self.ints)
        self.prev = None

    # ------------------------------------------------------------- a step
    def enlarged(self, i):
        bL, opsL = self.L[i]
        bR, opsR = self.R[i + 2]
        EL, chL, enlL = blocking_left_mixed(self.ints, bL, opsL, i, self.cut)
        ER, chR, enlR = blocking_right_mixed(self.ints, bR, opsR, i + 1, self.cut)
        return EL, assemble_all(enlL, EL, chL), ER, assemble_all(enlR, ER, chR)

    def predict(self, i, forward):
        """Guess for the step at bond i from the previous step's psi
        (None if there is no usable previous step).

        Moving right (previous step at bond i-1): psi lived on
        (L_{i-1} x s_{i-1}) x (s_i x R_{i+1}); projecting its left index on
        the kept states of L_i (phi = U^T psi) leaves L_i x (s_i x R_{i+1}),
        i.e. (L_i x s_i) x R_{i+1} with no sign (the product state is
        c_l c_n c_r |0> in either grouping), and each state of R_{i+1} is a
        combination of states of s_{i+1} x R_{i+2} (its stored basis V):
            psi'[(l, n), :] = phi[l, (n, r)] V^T.
        Moving left is the mirror image with psi V and the stored basis U of
        L_{i+1} over L_i x s_i."""
        if self.prev is None:
            return None
        pi, pfwd, px, play = self.prev
        if pi == i:  # turn of the sweep: same bond, same blocks
            return px
        bL_new, bR_new = self.L[i][0], self.R[i + 2][0]
        ELn, chLn = enlarged_left(bL_new)
        ERn, chRn = enlarged_right(bR_new)
        lay, size = psi_layout(ELn, ERn, self.Q)
        out = {qL: np.zeros((mL, mR)) for qL, qR, mL, mR, off in lay}
        qR_of = {qL: qR for qL, qR, mL, mR, off in lay}
        prev = psi_to_blocks(px, play)
        if forward and pfwd and pi == i - 1:
            U, V = self.UL[i], self.UR[i + 1]
            _, chR = enlarged_right(self.R[i + 1][0])
            bR1 = self.R[i + 1][0]
            row_of = {Q: {(qb, n): off for qb, n, off in lst} for Q, lst in chLn.items()}
            for QL, QR, mL, mR, off in play:
                if QL not in U:
                    continue
                phi = U[QL].T @ prev[QL]
                for qr, n, offc in chR[QR]:
                    QLn = qadd(QL, SITE_Q[n])
                    if QLn not in out or qR_of[QLn] != qr or qr not in V:
                        continue
                    r0 = row_of[QLn][(QL, n)]
                    out[QLn][r0:r0 + phi.shape[0], :] += phi[:, offc:offc + bR1.dim(qr)] @ V[qr].T
        elif not forward and not pfwd and pi == i + 1:
            V, U = self.UR[i + 2], self.UL[i + 1]
            _, chL = enlarged_left(self.L[i + 1][0])
            bL1 = self.L[i + 1][0]
            col_of = {Q: {(qb, n): off for qb, n, off in lst} for Q, lst in chRn.items()}
            for QL, QR, mL, mR, off in play:
                if QR not in V:
                    continue
                phi = prev[QL] @ V[QR]
                for ql, n, offc in chL[QL]:
                    QRn = qadd(QR, SITE_Q[n])
                    if ql not in out or qR_of[ql] != QRn or ql not in U:
                        continue
                    c0 = col_of[QRn][(QR, n)]
                    out[ql][:, c0:c0 + phi.shape[1]] += U[ql] @ phi[offc:offc + bL1.dim(ql), :]
        else:
            return None
        g = blocks_to_psi(out, lay, size)
        return g if np.linalg.norm(g) > 1e-12 else None

    def solve(self, i, step_id, EL, oL, ER, oR, guess=None):
        terms = mixed_terms(i + 1, self.K, self.cut)
        layout, size = psi_layout(EL, ER, self.Q)
        diag = heff_diagonal(layout, terms, oL, oR)
        if guess is not None:
            g = guess
        else:
            key = splitmix.stream_key(self.seed, splitmix.KEY_GUESS)
            g = splitmix.normal(key, (np.uint64(step_id) << np.uint64(32)) + np.arange(size, dtype=np.uint64))
        mv = lambda x: sigma_blocks(x, layout, terms, oL, oR)
        th, x, nmv, conv = davidson(mv, diag, g, **self.dav)
        return th, x, layout, nmv, conv

    def perturb(self, x, step_id):
        """Perturbative noise (the paper runs two-site DMRG with noise, Sec. III):
        the wavefunction handed to decimation is s x + noise * z / |z|, renormalized,
        with s = sign(x . z) (the solver's sign of x is arbitrary)
        with z seeded N(0,1) numbers (noise stream, counter (step_id << 32) + i),
        so that states the current wavefunction does not reach can enter the
        kept basis."""
        if self.noise == 0.0:
            return x
        key = splitmix.stream_key(self.seed, splitmix.KEY_NOISE)
        z = splitmix.normal(key, (np.uint64(step_id) << np.uint64(32)) + np.arange(len(x), dtype=np.uint64))
        sgn = -1.0 if x @ z < 0.0 else 1.0   # eigenvector sign is arbitrary: align x with z first
        y = sgn * x + self.noise * z / np.linalg.norm(z)
        return y / np.linalg.norm(y)

    @staticmethod
    def decimate(x, layout, M, keep_one_per_q=False):
        """Per-block SVD and global truncation. Returns (kept per q_L, U, V, discarded weight).
        keep_one_per_q: a block none of whose states made the global cut keeps its
        largest one as well (the paper keeps at least one state per quantum
        number, Sec. III), so the kept count may exceed M."""
        blocks = psi_to_blocks(x, layout)
        svd, cand = {}, []
        for qL, qR, mL, mR, off in layout:
            u, s, vt = np.linalg.svd(blocks[qL], full_matrices=False)
            svd[qL] = (u, s, vt, qR)
            cand += [(-float(sv), qL, k) for k, sv in enumerate(s)]
        cand.sort()
        keep = min(M, len(cand))
        kept = {}
        for _, qL, k in cand[:keep]:
            kept[qL] = kept.get(qL, 0) + 1
        disc = sum(c[0] ** 2 for c in cand[keep:])
        if keep_one_per_q:
            for qL, qR, mL, mR, off in layout:
                if kept.get(qL, 0) == 0 and min(mL, mR) > 0:
                    kept[qL] = 1
                    disc -= float(svd[qL][1][0]) ** 2
        return kept, svd, disc

    def step(self, i, forward, M, step_id):
        EL, oL, ER, oR = self.enlarged(i)
        th, x, layout, nmv, conv = self.solve(i, step_id, EL, oL, ER, oR, self.predict(i, forward))
        self.prev = (i, forward, x, layout)
        kept, svd, disc = self.decimate(self.perturb(x, step_id), layout, M, self.keep_one_per_q)
        if forward:
            U = {qL: fix_sign(svd[qL][0][:, :m]) for qL, m in kept.items()}
            nb = Basis(list(kept.items()))
            self.L[i + 1] = (nb, {k: transform(o, U, nb) for k, o in oL.items()})
            self.UL[i + 1] = U
        else:
            V, secs = {}, []
            for qL, m in kept.items():
                qR = svd[qL][3]
                V[qR] = fix_sign(svd[qL][2][:m, :].T)
                secs.append((qR, m))
            nb = Basis(secs)
            self.R[i + 1] = (nb, {k: transform(o, V, nb) for k, o in oR.items()})
            self.UR[i + 1] = V
        self.log.append(dict(i=i, forward=forward, M=M, energy=th, nmv=nmv,
                             converged=conv, discarded=disc, dim=len(x), kept=sum(kept.values())))
        return th, disc

    def sweep(self, M_schedule):
        """One entry of M_schedule per sweep (forward, backward, forward, ...).
        Returns (energies per sweep, max discarded weight per sweep)."""
        K = self.K
        energies, discs = [], []
        for s, M in enumerate(M_schedule):
            fwd = s % 2 == 0
            sites = range(0, K - 1) if fwd else range(K - 2, -1, -1)
            es, ds = [], []
            for i in sites:
                e, d = self.step(i, fwd, M, s * K + i)
                es.append(e)
                ds.append(d)
            energies.append(min(es))
            discs.append(max(ds))
        return energies, discs
