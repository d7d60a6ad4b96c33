"""Host logic of the blocking formulas, on the CPU: the library's own term
lists for an enlarged block (csrc/terms.cpp: NC left/right, CN left/right,
and the normal-to-complementary transformation in both directions), applied
by tests/host/blocking_check.cpp to exact Fock-space operators of the block,
must give the exact Fock-space operators of the enlarged block, operator by
operator (the same pin as the oracle's blocking formulas, Eq. blocked-ops)."""

import os
import shutil
import struct
import subprocess

import numpy as np
import pytest

from oracle.blocks import enlarged_left, enlarged_right
from oracle.nc import Integrals, fock_ops_exact
from synth import random_integrals
from test_oracle_nc import _enlarged_index_left, _enlarged_index_right

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def canonical_keys(nL, n, left, cn):
    """Operator keys in the library's canonical order (pairs over [0, nL) in
    NC form, over [nL, n) in CN form)."""
    keys = ["H"]
    if left:
        keys += [("cd", p) for p in range(nL)] + [("RL", p) for p in range(nL, n)]
    else:
        keys += [("d", p) for p in range(nL, n)] + [("RR", p) for p in range(nL)]
    lo, hi = (nL, n) if cn else (0, nL)
    normal = left != cn
    keys += [("A" if normal else "P", p, r) for p in range(lo, hi) for r in range(p + 1, hi)]
    keys += [("B" if normal else "Q", p, q) for p in range(lo, hi) for q in range(p, hi)]
    return keys


def _store(ops, keys, basis):
    """Flat store in the library's layout: operators in key order, blocks by
    ascending input sector, row-major."""
    parts = []
    for k in keys:
        op = ops[k]
        for q in basis.qs:
            if q in op.blocks:
                parts.append(np.ascontiguousarray(op.blocks[q]).ravel())
    return np.concatenate(parts) if parts else np.zeros(0)


def _dense(flat, keys, E, dqs):
    """Dense matrices over the enlarged basis E from a flat store."""
    out, off = {}, 0
    for k in keys:
        D = np.zeros((E.total, E.total))
        dq = dqs[k]
        for q in E.qs:
            qo = (q[0] + dq[0], q[1] + dq[1])
            if not E.has(qo):
                continue
            r, c = E.dim(qo), E.dim(q)
            i0, j0 = E.offsets[E.index[qo]], E.offsets[E.index[q]]
            D[i0:i0 + r, j0:j0 + c] = flat[off:off + r * c].reshape(r, c)
            off += r * c
        out[k] = D
    assert off == len(flat)
    return out


@pytest.fixture(scope="module")
def checker(tmp_path_factory):
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("no C++ compiler")
    out = str(tmp_path_factory.mktemp("blk") / "blocking_check")
    csrc = os.path.join(ROOT, "paper_2103_09976_gb300", "csrc")
    subprocess.run([gxx, "-O2", "-std=c++17", "-I", csrc, os.path.join(ROOT, "tests", "host", "blocking_check.cpp"),
                    os.path.join(csrc, "terms.cpp"), os.path.join(csrc, "model.cpp"), "-o", out], check=True)
    return out


CASES = [("L", "nc", "nc"), ("L", "nc", "cn"), ("L", "cn", "cn"),
         ("R", "nc", "nc"), ("R", "cn", "nc"), ("R", "cn", "cn")]


@pytest.mark.parametrize("side,src,dst", CASES)
def test_host_blocking_equals_fock_operators(checker, tmp_path, side, src, dst):
    K = 4
    t, v = random_integrals(K, 17)
    ints = Integrals(t, v)
    n = 2 * K
    left = side == "L"
    for site in (range(0, K) if left else range(0, K - 1)):
        if left:
            if site == 0 and src == "cn":
                continue  # an empty left block is only ever in NC form
            bmodes, emodes = list(range(2 * site)), list(range(2 * site + 2))
            nLb, nE = 2 * site, 2 * site + 2
        else:
            if site == K - 1:
                continue
            bmodes, emodes = list(range(2 * site + 2, n)), list(range(2 * site, n))
            nLb, nE = 2 * site + 2, 2 * site
        if not bmodes:
            continue
        bB, pB, oB = fock_ops_exact(ints, bmodes, side, src)
        bX, pX, oX = fock_ops_exact(ints, emodes, side, dst)
        keys_b = canonical_keys(nLb, n, left, src == "cn")
        keys_e = canonical_keys(nE, n, left, dst == "cn")
        assert set(keys_b) == set(oB) and set(keys_e) == set(oX)
        store = _store(oB, keys_b, bB)
        inp = tmp_path / "in.bin"
        with open(inp, "wb") as f:
            f.write(struct.pack("6i", K, 0 if left else 1, site, int(src == "cn"), int(dst == "cn"), len(bB.qs)))
            for q, d in zip(bB.qs, bB.dims):
                f.write(struct.pack("3i", q[0], q[1], d))
            f.write(np.asarray(t, dtype=np.float64).tobytes())
            f.write(np.asarray(v, dtype=np.float64).tobytes())
            f.write(store.tobytes())
        outp = tmp_path / "out.bin"
        subprocess.run([checker, str(inp), str(outp)], check=True)
        raw = open(outp, "rb").read()
        cnt = struct.unpack("q", raw[:8])[0]
        flat = np.frombuffer(raw[8:], dtype=np.float64, count=cnt)
        E, ch = enlarged_left(bB) if left else enlarged_right(bB)
        got = _dense(flat, keys_e, E, {k: oX[k].dq for k in keys_e})
        pos = np.argsort(pX)[_enlarged_index_left(E, ch, bB, pB, nLb) if left else _enlarged_index_right(E, ch, bB, pB)]
        for k in keys_e:
            ref = oX[k].to_dense()[np.ix_(pos, pos)]
            assert np.abs(got[k] - ref).max() < 1e-12, (side, src, dst, site, k)
