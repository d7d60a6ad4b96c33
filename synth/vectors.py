"""Seeded random vectors (wavefunction guesses and sigma inputs)."""

import numpy as np


def random_unit_vector(n, seed):
    """N(0,1) entries from numpy.random.default_rng(seed), scaled to unit 2-norm."""
    x = np.random.default_rng(seed).standard_normal(n)
    nrm = np.linalg.norm(x)
    return x / nrm if nrm > 0 else x
