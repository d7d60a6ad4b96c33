"""Host logic of the sigma work lists, on the CPU: the library's own C++
(tests/host/plan_check.cpp linked against csrc/model.cpp, no CUDA calls)
builds the operator tables, the NC or CN term list, the task list and the
tensor-core plan; its psi layout must equal the oracle's exactly, its
product count and algorithmic flops the oracle's independent count over the
same sectors (oracle.sigma.sigma_flops; the plan holds every product once per
128 x 128 tile of its output block), its sub-Hamiltonian rank of every term
the oracle's (nc_term_rank),
and both work lists must pass their structural checks (FP64: 32 x 256 tiles
whose items split each block's tasks in order; tensor-core plan: every task
once per tile, units in order, 128 x 128 tiles of every output block,
scratch slots, schedule, records)."""

import json
import os
import shutil
import subprocess

import pytest

from oracle.blocks import Basis, qadd
from oracle.cn import cn_terms
from oracle.nc import nc_terms, spin
from oracle.sigma import nc_term_rank, psi_layout, sigma_flops, synthetic_op_specs
from synth import gaussian_sector_dims, mirrored_sectors

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def checker(tmp_path_factory):
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("no C++ compiler")
    out = str(tmp_path_factory.mktemp("plan") / "plan_check")
    csrc = os.path.join(ROOT, "paper_2103_09976_gb300", "csrc")
    subprocess.run([gxx, "-O2", "-std=c++17", "-pthread", "-I", csrc, os.path.join(ROOT, "tests", "host", "plan_check.cpp"),
                    os.path.join(csrc, "model.cpp"), "-o", out], check=True)
    return out


def _dq_maps(nL, n, cn):
    if not cn:
        specs = synthetic_op_specs(nL, n)
        return ({k: dq for side, k, dq, sym in specs if side == "L"},
                {k: dq for side, k, dq, sym in specs if side == "R"})
    L, R = range(nL), range(nL, n)
    dqL = {"H": (0, 0)}
    dqL.update({("cd", p): (1, spin(p)) for p in L})
    dqL.update({("RL", p): (-1, -spin(p)) for p in R})
    dqL.update({("P", p, r): (-2, -spin(p) - spin(r)) for p in R for r in R if p < r})
    dqL.update({("Q", p, q): (0, -(spin(p) - spin(q))) for p in R for q in R if p <= q})
    dqR = {"H": (0, 0)}
    dqR.update({("d", p): (-1, -spin(p)) for p in R})
    dqR.update({("RR", p): (-1, -spin(p)) for p in L})
    dqR.update({("A", p, r): (2, spin(p) + spin(r)) for p in R for r in R if p < r})
    dqR.update({("B", p, q): (0, spin(p) - spin(q)) for p in R for q in R if p <= q})
    return dqL, dqR


def _products(layout, terms, dqL, dqR, weight=None):
    """Number of (term, psi block) products; with weight, each product counts
    weight[output block's left sector] times."""
    blk = {qL: qR for qL, qR, mL, mR, off in layout}
    count = 0
    for kl, tl, kr, tr, c in terms:
        dx = (0, 0) if kl is None else (dqL[kl] if not tl else (-dqL[kl][0], -dqL[kl][1]))
        dy = (0, 0) if kr is None else (dqR[kr] if not tr else (-dqR[kr][0], -dqR[kr][1]))
        for qL, qR in blk.items():
            qLo = qadd(qL, dx)
            if qLo in blk and blk[qLo] == qadd(qR, dy):
                count += 1 if weight is None else weight[qLo]
    return count


# sectors with blocks above 128 rows / columns: several output tiles per block
# and psi blocks wider than one 128-column pass
BIG = [(3, -1, 40), (3, 1, 40), (4, -2, 129), (4, 0, 300), (4, 2, 130), (5, -1, 64), (5, 1, 200), (6, 0, 17)]


@pytest.mark.parametrize("nsp,ntot,two_sz,M,cn", [(6, 12, 0, 150, False), (6, 12, 0, 150, True),
                                                  (8, 9, 1, 300, True), (54, 30, 0, 400, False),
                                                  (4, 8, 0, None, False), (4, 8, 0, None, True)])
def test_task_list_and_plan_match_the_oracle_count(checker, tmp_path, nsp, ntot, two_sz, M, cn):
    if M is None:
        left = BIG
        right = sorted((ntot - n, two_sz - s, d) for n, s, d in BIG)
    else:
        left = gaussian_sector_dims(M, n_spatial=nsp, n_tot=ntot, two_sz_tot=two_sz)
        right = mirrored_sectors(left, n_tot=ntot, two_sz_tot=two_sz)
    path = tmp_path / "sectors.txt"
    with open(path, "w") as f:
        f.write(f"{len(left)} {len(right)}\n")
        for s in list(left) + list(right):
            f.write(" ".join(str(int(x)) for x in s) + "\n")
    nL, n = 2 * nsp, 4 * nsp
    out = subprocess.run([checker, str(path), str(nL), str(n), str(ntot), str(two_sz), "cn" if cn else "nc"],
                         check=True, capture_output=True, text=True).stdout
    got = json.loads(out)
    assert got["errors"] == []
    bL = Basis([((a, b), d) for a, b, d in left])
    bR = Basis([((a, b), d) for a, b, d in right])
    layout, size = psi_layout(bL, bR, (ntot, two_sz))
    terms = cn_terms(nL, n) if cn else nc_terms(nL, n)
    dqL, dqR = _dq_maps(nL, n, cn)
    assert got["psi_size"] == size and got["blocks"] == len(layout) and got["terms"] == len(terms)
    # sector bookkeeping: the psi layout is bit-identical to the oracle's
    assert got["layout"] == [[qL[0], qL[1], qR[0], qR[1], mL, mR, off] for qL, qR, mL, mR, off in layout]
    assert got["tasks"] == _products(layout, terms, dqL, dqR)
    tiles = {qL: ((mL + 127) // 128) * ((mR + 127) // 128) for qL, qR, mL, mR, off in layout}
    assert got["plan_tasks"] == _products(layout, terms, dqL, dqR, tiles)
    ref = sigma_flops(layout, terms, dqL, dqR, bL, bR)
    assert abs(got["flops"] - ref) <= 1e-12 * ref
    # sub-Hamiltonian ranks of the terms (Eqs. proc-def-nc / proc-def-cn), 3 ranks
    assert got["ranks3"] == [nc_term_rank(t, 3) for t in terms]


def test_bench_size_plan_stays_in_bounds(checker, tmp_path):
    """The middle-bond plan the bench times (K=108, N=30, 2Sz=0, M=2000: 364k
    units of stacked terms): every bulk copy of the tensor-core kernel, in both
    producer settings, lands inside its stage and reads inside the split
    arrays, and every MMA operand read stays inside its stage or term region;
    the work list and the plan cover the same products."""
    left = gaussian_sector_dims(2000, n_spatial=54, n_tot=30, two_sz_tot=0)
    right = mirrored_sectors(left, n_tot=30, two_sz_tot=0)
    path = tmp_path / "sectors.txt"
    with open(path, "w") as f:
        f.write(f"{len(left)} {len(right)}\n")
        for s in list(left) + list(right):
            f.write(" ".join(str(int(x)) for x in s) + "\n")
    out = subprocess.run([checker, str(path), "108", "216", "30", "0", "nc"], check=True, capture_output=True,
                         text=True).stdout
    got = json.loads(out)
    assert got["errors"] == []
    assert got["terms"] == 23654 and got["psi_size"] == 106004
    assert got["units"] > 300000 and got["stages"] > got["units"]
