"""Pins of the oracle's counter-based generator (SplitMix64 + Box-Muller)."""

import os

import numpy as np

from oracle import splitmix

GOLD = os.path.join(os.path.dirname(__file__), "golden", "splitmix64_seed1234567.txt")


def test_splitmix64_published_sequence():
    want = [int(x) for x in open(GOLD) if x.strip() and not x.startswith("#")]
    got = splitmix.splitmix64(1234567, np.arange(5))
    assert [int(x) for x in got] == want


def test_counter_form_equals_sequential_state():
    # The counter form must equal running the generator's state forward.
    key = 0xDEADBEEF
    state = key
    seq = []
    for _ in range(10):
        state = (state + 0x9E3779B97F4A7C15) & 0xFFFFFFFFFFFFFFFF
        seq.append(int(splitmix.mix64(np.uint64(state))))
    assert seq == [int(x) for x in splitmix.splitmix64(key, np.arange(10))]


def test_uniform_range_and_normal_moments():
    u = splitmix.uniform01(7, np.arange(200000))
    assert u.min() > 0.0 and u.max() <= 1.0
    z = splitmix.normal(11, np.arange(400000))
    assert abs(z.mean()) < 0.01
    assert abs(z.var() - 1.0) < 0.01
    # fourth moment of a standard normal is 3
    assert abs((z ** 4).mean() - 3.0) < 0.05
