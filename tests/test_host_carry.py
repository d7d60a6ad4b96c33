"""Host logic of the wavefunction carry between sweep steps, on the CPU: the
library's own job lists (csrc/terms.cpp carry_jobs), applied by
tests/host/carry_check.cpp to the oracle's previous psi and stored bases,
must give the oracle's carried start vector (oracle.dmrg.PlainDMRG.predict)
at every step of truncated sweeps in both directions, NC and mixed NC/CN."""

import os
import shutil
import struct
import subprocess

import numpy as np
import pytest

from oracle.dmrg import PlainDMRG
from synth import random_integrals

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def checker(tmp_path_factory):
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("no C++ compiler")
    out = str(tmp_path_factory.mktemp("carry") / "carry_check")
    csrc = os.path.join(ROOT, "paper_2103_09976_gb300", "csrc")
    subprocess.run([gxx, "-O2", "-std=c++17", "-I", csrc, os.path.join(ROOT, "tests", "host", "carry_check.cpp"),
                    os.path.join(csrc, "terms.cpp"), os.path.join(csrc, "model.cpp"), "-o", out], check=True)
    return out


def _basis(f, b):
    f.write(struct.pack("i", len(b.qs)))
    for q, d in zip(b.qs, b.dims):
        f.write(struct.pack("3i", q[0], q[1], d))


def _carried(checker, path, d, i, forward):
    """psi' from the library's carry jobs, for the step at bond i."""
    pi, pfwd, px, play = d.prev
    if forward:
        pL, pR, nL, nR = d.L[i - 1][0], d.R[i + 1][0], d.L[i][0], d.R[i + 2][0]
        lb, lu, rb, ru = d.L[i][0], d.UL[i], d.R[i + 1][0], d.UR[i + 1]
    else:
        pL, pR, nL, nR = d.L[i + 1][0], d.R[i + 3][0], d.L[i][0], d.R[i + 2][0]
        lb, lu, rb, ru = d.L[i + 1][0], d.UL[i + 1], d.R[i + 2][0], d.UR[i + 2]
    inp, outp = str(path / "in.bin"), str(path / "out.bin")
    with open(inp, "wb") as f:
        f.write(struct.pack("3i", int(forward), d.Q[0], d.Q[1]))
        for b in (pL, pR, nL, nR):
            _basis(f, b)
        for b, U in ((lb, lu), (rb, ru)):
            _basis(f, b)
            for q in b.qs:
                f.write(np.ascontiguousarray(U[q], dtype=np.float64).tobytes())
        f.write(np.asarray(px, dtype=np.float64).tobytes())
    subprocess.run([checker, inp, outp], check=True)
    raw = open(outp, "rb").read()
    n = struct.unpack("q", raw[:8])[0]
    return np.frombuffer(raw[8:], dtype=np.float64, count=n)


@pytest.mark.parametrize("cut", [None, 2])
def test_carried_guess_equals_the_oracle(checker, tmp_path, cut):
    K, N, s, M = 5, 5, 1, 8
    t, v = random_integrals(K, 23)
    d = PlainDMRG(t, v, N, s, seed=4, dav_tol=1e-12, cut=cut)
    d.build_blocks(M)
    checked = 0
    for sweep in range(3):
        fwd = sweep % 2 == 0
        for i in (range(0, K - 1) if fwd else range(K - 2, -1, -1)):
            g = d.predict(i, fwd)
            if g is not None and d.prev[0] != i:
                got = _carried(checker, tmp_path, d, i, fwd)
                assert got.shape == g.shape
                assert np.abs(got - g).max() <= 1e-13 * max(1.0, np.abs(g).max()), (sweep, i)
                checked += 1
            d.step(i, fwd, M, sweep * K + i)
    assert checked == 3 * (K - 2)
