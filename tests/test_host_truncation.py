"""Host logic of the global truncation, on the CPU: the library's
select_kept (csrc/terms.cpp), given the singular values the oracle's
decimation computes, keeps the oracle's states per quantum number and
discards the same weight (reading c8: sort by value descending, q_L
ascending, index ascending, keep min(M, count) including zeros; c20: one
state per quantum number on request), including exact ties across blocks."""

import json
import os
import shutil
import subprocess

import numpy as np
import pytest

from oracle.blocks import Basis
from oracle.dmrg import PlainDMRG
from oracle.sigma import blocks_to_psi, psi_layout

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def checker(tmp_path_factory):
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("no C++ compiler")
    out = str(tmp_path_factory.mktemp("trunc") / "truncation_check")
    csrc = os.path.join(ROOT, "paper_2103_09976_gb300", "csrc")
    subprocess.run([gxx, "-O2", "-std=c++17", "-I", csrc, os.path.join(ROOT, "tests", "host", "truncation_check.cpp"),
                    os.path.join(csrc, "terms.cpp"), os.path.join(csrc, "model.cpp"), "-o", out], check=True)
    return out


def _layout():
    bL = Basis([((2, 0), 3), ((3, -1), 2), ((3, 1), 4), ((4, 0), 5)])
    bR = Basis([((2, 0), 5), ((3, -1), 4), ((3, 1), 2), ((4, 0), 3)])
    return psi_layout(bL, bR, (6, 0))


@pytest.mark.parametrize("kind", ["random", "ties"])
@pytest.mark.parametrize("M,keep_one", [(1, False), (3, False), (5, True), (7, False), (2, True), (40, False)])
def test_kept_states_equal_the_oracle(checker, kind, M, keep_one):
    layout, size = _layout()
    rng = np.random.default_rng(M + 10 * keep_one)
    blocks = {}
    for qL, qR, mL, mR, off in layout:
        if kind == "random":
            blocks[qL] = rng.standard_normal((mL, mR))
        else:  # diagonal blocks: exactly representable singular values, equal across blocks
            B = np.zeros((mL, mR))
            vals = [0.5, 0.5, 0.25, 0.0, 0.125][:min(mL, mR)]
            for i, x in enumerate(vals):
                B[i, i] = x
            blocks[qL] = B
    x = blocks_to_psi(blocks, layout, size)
    kept, svd, disc = PlainDMRG.decimate(x, layout, M, keep_one)
    inp = f"{len(layout)}\n" + "\n".join(
        f"{qL[0]} {qL[1]} {len(svd[qL][1])} " + " ".join(repr(float(v)) for v in svd[qL][1]) for qL, *_ in layout)
    out = subprocess.run([checker, str(M), str(int(keep_one))], input=inp, capture_output=True, text=True,
                         check=True).stdout
    got = json.loads(out)
    want = [kept.get(qL, 0) for qL, *_ in layout]
    assert got["kept"] == want, (got["kept"], want)
    assert abs(got["discarded"] - disc) <= 1e-15 * max(1.0, abs(disc))
