"""Random real one- and two-electron integrals with the symmetry of the
ab initio Hamiltonian (Appendix B, Eq. qc-hamil and the 8-fold symmetry
conditions that follow it).

Conventions:
  * t is K x K, real symmetric.
  * v is K x K x K x K in chemist's notation v[i,j,k,l] = (ij|kl), entering
    H as 1/2 sum v_ijkl a+_{i s} a+_{k s'} a_{l s'} a_{j s}, with
    v_ijkl = v_jikl = v_ijlk = v_klij.

Drawing order (fixed so that every consumer sees the same arrays):
  1. t: the upper triangle (i <= j) in row-major order, N(0, 1), mirrored.
  2. v: unique tuples i >= j, k >= l, (ij) >= (kl) in lexicographic order of
     (i, j, k, l), N(0, scale_v^2), then expanded to all 8 symmetric images.
Both are drawn from one numpy.random.default_rng(seed) stream, t first.
"""

import numpy as np


def _pair_list(K):
    return [(i, j) for i in range(K) for j in range(i + 1)]


def random_integrals(K, seed, scale_t=1.0, scale_v=0.1, decay=None):
    """Return (t, v) as float64 arrays of shapes (K, K) and (K, K, K, K).

    decay: if given, t_ij is multiplied by exp(-|i-j|/decay) and v_ijkl by
    exp(-(|i-j| + |k-l|)/decay), which keeps the 8-fold symmetry.
    """
    rng = np.random.default_rng(seed)
    t = np.zeros((K, K))
    iu = np.triu_indices(K)
    t[iu] = scale_t * rng.standard_normal(len(iu[0]))
    t = t + t.T - np.diag(np.diag(t))

    pairs = _pair_list(K)
    npair = len(pairs)
    a_idx, b_idx = np.tril_indices(npair)  # a >= b, row-major = lexicographic
    vals = scale_v * rng.standard_normal(len(a_idx))
    P = np.array(pairs, dtype=np.int64)
    i, j = P[a_idx, 0], P[a_idx, 1]
    k, l = P[b_idx, 0], P[b_idx, 1]
    v = np.zeros((K, K, K, K))
    for (w, x, y, z) in ((i, j, k, l), (j, i, k, l), (i, j, l, k), (j, i, l, k),
                         (k, l, i, j), (l, k, i, j), (k, l, j, i), (l, k, j, i)):
        v[w, x, y, z] = vals

    if decay is not None:
        idx = np.arange(K)
        d = np.abs(idx[:, None] - idx[None, :]).astype(np.float64)
        t = t * np.exp(-d / decay)
        v = v * np.exp(-(d[:, :, None, None] + d[None, None, :, :]) / decay)
    return t, v


def femoco_like_integrals(K=76, seed=2, decay=8.0):
    """Integrals for the FeMoco-shaped sweep workload: the random scales of
    random_integrals with couplings that decay as exp(-|p-q|/8)."""
    return random_integrals(K, seed, decay=decay)
