"""Native serving loop (dmrg_server_*): every result is bitwise the same
alone and in the mix, equals a direct dmrg_davidson call, and admission
keeps the device footprint of concurrently running solves within the
budget."""

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

# (id, K spatial, N, 2Sz, M, seed, precision name)
REQS = [(0, 12, 8, 0, 60, 11, "FP64"), (1, 16, 10, 0, 120, 12, "FP64"), (2, 12, 7, 1, 80, 13, "BF16X3"),
        (3, 20, 12, 0, 200, 14, "FP64"), (4, 16, 9, 1, 150, 15, "FP16X2"), (5, 12, 8, 0, 60, 16, "BF16X2")]
TOL, MAX_ITER = 1e-9, 40


def _submit(capi, srv, r):
    from paper_2103_09976_gb300.serve import request_sectors
    i, K, N, s, M, seed, prec = r
    left, right = request_sectors(K, N, s, M)
    capi.dmrg_server_submit(srv, i, K, 2 * K, N, s, left, right, seed, getattr(capi, "DMRG_" + prec), MAX_ITER, TOL)


def _collect(capi, srv, n):
    out = {}
    for _ in range(2000):
        for res in capi.dmrg_server_poll(srv, 16, wait_ms=50):
            out[res["id"]] = res
        if len(out) == n:
            return out
    raise AssertionError("server did not finish")


def test_alone_equals_mixed_equals_direct():
    from paper_2103_09976_gb300 import capi
    from paper_2103_09976_gb300.serve import request_sectors
    alone = {}
    srv = capi.dmrg_server_create(0, 1, 64 << 30)
    try:
        for r in REQS:
            _submit(capi, srv, r)
            alone.update(_collect(capi, srv, 1))
    finally:
        capi.dmrg_server_destroy(srv)
    srv = capi.dmrg_server_create(0, 4, 64 << 30)
    try:
        for r in REQS:
            _submit(capi, srv, r)
        mixed = _collect(capi, srv, len(REQS))
    finally:
        capi.dmrg_server_destroy(srv)
    assert len({res["slot"] for res in mixed.values()}) > 1          # solves ran on several slots
    for r in REQS:
        a, m = alone[r[0]], mixed[r[0]]
        assert a["status"] == m["status"] == capi.DMRG_OK
        assert a["energy"] == m["energy"] and a["iters"] == m["iters"], (r, a, m)
    # the first request directly through dmrg_davidson
    i, K, N, s, M, seed, prec = REQS[3]
    left, right = request_sectors(K, N, s, M)
    ctx = capi.dmrg_create(device=0, seed=seed, dav_max_iter=MAX_ITER)
    try:
        capi.dmrg_load_synthetic(ctx, K, 2 * K, N, s, left, right, seed)
        e, it, conv = capi.dmrg_davidson(ctx, -1, None, TOL)
    finally:
        capi.dmrg_destroy(ctx)
    assert e == alone[i]["energy"] and it == alone[i]["iters"]


def test_admission_respects_budget():
    from paper_2103_09976_gb300 import capi
    srv = capi.dmrg_server_create(0, 4, 64 << 30)
    try:
        for r in REQS:
            _submit(capi, srv, r)
        first = _collect(capi, srv, len(REQS))
    finally:
        capi.dmrg_server_destroy(srv)
    bytes_of = {k: v["bytes"] for k, v in first.items()}
    budget = int(1.2 * max(bytes_of.values()))
    srv = capi.dmrg_server_create(0, 4, budget)
    try:
        for r in REQS:
            _submit(capi, srv, r)
        res = _collect(capi, srv, len(REQS))
        with pytest.raises(capi.DMRGError) as ei:
            big = (99, 24, 12, 0, 1000, 1, "FP64")
            _submit(capi, srv, big)
        assert ei.value.status == capi.DMRG_ENOMEM
    finally:
        capi.dmrg_server_destroy(srv)
    events = sorted([(v["t_admit"], v["bytes"]) for v in res.values()] +
                    [(v["t_done"], -v["bytes"]) for v in res.values()], key=lambda x: (x[0], x[1]))
    used = 0
    for _, b in events:
        used += b
        assert used <= budget
    assert all(v["status"] == capi.DMRG_OK for v in res.values())
