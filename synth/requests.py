"""Seeded stream of Davidson-solve requests for the serving workload.

Each request has an arrival time (Poisson process), an orbital count K, an
electron count N ~ U[K/2, K], 2Sz = N mod 2, a bond dimension M and a seed for
its integrals.
"""

import numpy as np

K_CHOICES = (24, 36, 54, 76, 108)
M_CHOICES = (250, 500, 1000, 2000, 4000)


def poisson_requests(n_req=256, rate_per_s=1.0, seed=5, k_choices=K_CHOICES,
                     m_choices=M_CHOICES):
    rng = np.random.default_rng(seed)
    gaps = rng.exponential(1.0 / rate_per_s, size=n_req)
    arrive = np.cumsum(gaps) - gaps[0]
    out = []
    for r in range(n_req):
        K = int(rng.choice(k_choices))
        N = int(rng.integers(K // 2, K + 1))
        M = int(rng.choice(m_choices))
        out.append({"id": r, "t_arrive": float(arrive[r]), "K": K, "N": N,
                    "two_sz": N % 2, "M": M, "seed": 1000 + r})
    return out
