"""Counter-based random numbers for synthetic operator blocks (oracle side).

SplitMix64 (G. Steele, D. Lea, C. Flood, "Fast splittable pseudorandom number
generators", OOPSLA 2014; finalizer constants as in S. Vigna's public-domain
splitmix64.c). Used here as a counter-based generator: the c-th output of a
generator started from state `key` is

    mix(key + (c + 1) * 0x9E3779B97F4A7C15)   (mod 2^64)

with mix(z) = z ^= z>>30; z *= 0xBF58476D1CE4E5B9; z ^= z>>27;
z *= 0x94D049BB133111EB; z ^= z>>31.

Uniform in (0, 1]: u = ((x >> 11) + 1) * 2^-53.
Standard normal for counter g (Box-Muller, cosine branch):
    z = sqrt(-2 ln u(2g)) * cos(2 pi u(2g+1)).

Pinned by tests/test_oracle_rng.py (published SplitMix64 output sequence,
moments of the normal draws). The CUDA library implements the same published
definition independently.
"""

import numpy as np

GAMMA = np.uint64(0x9E3779B97F4A7C15)
M1 = np.uint64(0xBF58476D1CE4E5B9)
M2 = np.uint64(0x94D049BB133111EB)


def mix64(z):
    z = np.asarray(z, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * M1
        z = (z ^ (z >> np.uint64(27))) * M2
    return z ^ (z >> np.uint64(31))


def splitmix64(key, counters):
    """Outputs number counters+1 of SplitMix64 seeded with `key` (vectorised)."""
    c = np.asarray(counters, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(key) + (c + np.uint64(1)) * GAMMA
    return mix64(z)


def uniform01(key, counters):
    x = splitmix64(key, counters)
    return ((x >> np.uint64(11)).astype(np.float64) + 1.0) * (2.0 ** -53)


def normal(key, g):
    """Standard normal number for flat counter(s) g."""
    g = np.asarray(g, dtype=np.uint64)
    u1 = uniform01(key, np.uint64(2) * g)
    u2 = uniform01(key, np.uint64(2) * g + np.uint64(1))
    return np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * np.pi * u2)


# Stream keys. Each independent random stream of the method derives its key
# from the user seed by XOR with one of these constants.
KEY_OPS = 0x0000000000000000
KEY_MPS = 0x4D50535F494E4954  # "MPS_INIT"
KEY_GUESS = 0x4755455353505349  # "GUESSPSI"
KEY_NOISE = 0x4E4F495345505349  # "NOISEPSI"


def stream_key(seed, which):
    return (int(seed) ^ int(which)) & 0xFFFFFFFFFFFFFFFF
