"""Sector dimension lists for the synthetic middle-bond sigma workload.

A side basis of total dimension M is spread over quantum numbers
q = (N, 2Sz) with weights of a 2-D Gaussian about (N0, 0): sigma_N = 3,
sigma_2Sz = 2. A sector (N, s) is admissible when it can pair with the
mirrored right sector (N_tot - N, -s) inside n_spatial orbitals per side:
0 <= N <= N_tot, s = N (mod 2), |s| <= min(N, N_tot - N, 2 n_spatial - N).
Dimensions come from largest-remainder rounding of M * w / sum(w) (ties by
ascending (N, s)); zero-dimension sectors are dropped.
"""

import numpy as np


def gaussian_sector_dims(M, n_spatial=54, n_tot=30, two_sz_tot=0,
                         center=None, sigma_n=3.0, sigma_s=2.0):
    """Return a list of (N, 2Sz, dim), ascending in (N, 2Sz), with sum(dim) == M."""
    if center is None:
        center = n_tot / 2.0
    cand = []
    for n in range(0, n_tot + 1):
        nr = n_tot - n
        if n > 2 * n_spatial or nr > 2 * n_spatial:
            continue
        smax = min(n, 2 * n_spatial - n)
        for s in range(-smax, smax + 1):
            if (s - n) % 2 != 0:
                continue
            sr = two_sz_tot - s
            srmax = min(nr, 2 * n_spatial - nr)
            if abs(sr) > srmax or (sr - nr) % 2 != 0:
                continue
            cand.append((n, s))
    w = np.array([np.exp(-(n - center) ** 2 / (2 * sigma_n ** 2)
                         - (s - two_sz_tot / 2.0) ** 2 / (2 * sigma_s ** 2))
                  for n, s in cand])
    exact = M * w / w.sum()
    base = np.floor(exact).astype(np.int64)
    rem = exact - base
    short = int(M - base.sum())
    order = sorted(range(len(cand)), key=lambda a: (-rem[a], cand[a]))
    for a in order[:short]:
        base[a] += 1
    out = [(n, s, int(d)) for (n, s), d in zip(cand, base) if d > 0]
    out.sort()
    assert sum(d for _, _, d in out) == M
    return out


def mirrored_sectors(left, n_tot=30, two_sz_tot=0):
    """Right-side sector list paired with `left`: (N_tot - N, 2Sz_tot - s), same dim."""
    right = [(n_tot - n, two_sz_tot - s, d) for n, s, d in left]
    right.sort()
    return right
