"""Serving workload: a Poisson stream of Davidson solves through the
library's native serving loop (dmrg_server_*), reporting p50/p99 latency
and solves/s.

Each request is a middle-bond problem of K spatial orbitals (K/2 per side,
K spin orbitals per side), N electrons, 2Sz = N mod 2 and bond dimension M,
with synthetic N(0,1) operator blocks seeded per request; latency is
completion time minus arrival time.

    python -m paper_2103_09976_gb300.serve --requests 48 --rate 0

With --rate auto the stream runs twice: first with every request arriving
at once (the burst measures the capacity in solves/s), then as a Poisson
stream at 80% of that capacity. The full request mix (256 solves, K in
{24, 36, 54, 76, 108}, M in {250, 500, 1000, 2000, 4000}):

    python -m paper_2103_09976_gb300.serve --requests 256 --rate auto \
        --k 24,36,54,76,108 --m 250,500,1000,2000,4000
"""

import argparse
import json
import time

import numpy as np

from . import capi


def request_sectors(K, N, two_sz, M):
    from synth import gaussian_sector_dims, mirrored_sectors
    left = gaussian_sector_dims(M, n_spatial=K // 2, n_tot=N, two_sz_tot=two_sz)
    right = mirrored_sectors(left, n_tot=N, two_sz_tot=two_sz)
    return left, right


def run_stream(requests, n_slots=4, budget_bytes=160 << 30, prec=capi.DMRG_FP16X2, tol=1e-8, max_iter=60,
               device=0, rate_scale=1.0):
    """Submit `requests` (dicts from synth.requests.poisson_requests) at their
    arrival times (scaled by rate_scale; 0 = all at once) and collect results."""
    srv = capi.dmrg_server_create(device, n_slots, budget_bytes)
    results, rejected = {}, {}
    peak = [0, 0]  # largest device bytes admitted at once, most solves running at once
    try:
        t0 = time.perf_counter()
        pending = sorted(requests, key=lambda r: r["t_arrive"])
        submitted = 0
        while len(results) + len(rejected) < len(requests):
            now = time.perf_counter() - t0
            while submitted < len(pending) and pending[submitted]["t_arrive"] * rate_scale <= now:
                r = pending[submitted]
                left, right = request_sectors(r["K"], r["N"], r["two_sz"], r["M"])
                try:
                    capi.dmrg_server_submit(srv, r["id"], r["K"], 2 * r["K"], r["N"], r["two_sz"], left, right,
                                            r["seed"], prec, max_iter, tol)
                except capi.DMRGError as e:
                    rejected[r["id"]] = str(e)
                submitted += 1
            for res in capi.dmrg_server_poll(srv, 64, wait_ms=5):
                results[res["id"]] = res
            _, running, in_use = capi.dmrg_server_pending(srv)
            peak[0] = max(peak[0], in_use)
            peak[1] = max(peak[1], running)
    finally:
        capi.dmrg_server_destroy(srv)
    run_stream.peak_bytes, run_stream.peak_running = peak
    return results, rejected


def summarize(results, requests):
    by_id = {r["id"]: r for r in requests}
    lat = np.array([res["t_done"] - res["t_submit"] for res in results.values()])
    span = max(res["t_done"] for res in results.values()) - min(res["t_submit"] for res in results.values())
    return {"solves": len(results), "p50_s": float(np.percentile(lat, 50)), "p99_s": float(np.percentile(lat, 99)),
            "solves_per_s": len(results) / span if span > 0 else None,
            "ok": sum(1 for r in results.values() if r["status"] == capi.DMRG_OK),
            "converged": sum(1 for r in results.values() if r["converged"]),
            "mean_load_s": float(np.mean([r["t_loaded"] - r["t_admit"] for r in results.values()])),
            "mean_solve_s": float(np.mean([r["t_done"] - r["t_loaded"] for r in results.values()])),
            "mix": sorted({(by_id[i]["K"], by_id[i]["M"]) for i in results})}


def main():
    from synth.requests import poisson_requests
    ap = argparse.ArgumentParser()
    ap.add_argument("--requests", type=int, default=48)
    ap.add_argument("--rate", default="4.0",
                    help="arrivals per second (0 = all at once; auto = burst, then Poisson at 80%% of its rate)")
    ap.add_argument("--slots", type=int, default=4)
    ap.add_argument("--budget-gb", type=float, default=160.0)
    ap.add_argument("--k", default="24,36,54")
    ap.add_argument("--m", default="250,500,1000")
    ap.add_argument("--max-iter", type=int, default=60)
    args = ap.parse_args()
    ks = tuple(int(x) for x in args.k.split(","))
    ms = tuple(int(x) for x in args.m.split(","))
    budget = int(args.budget_gb * (1 << 30))

    def phase(rate):
        reqs = poisson_requests(args.requests, rate_per_s=max(rate, 1e-9), seed=5 if rate == 0 else 6,
                                k_choices=ks, m_choices=ms)
        res, rej = run_stream(reqs, n_slots=args.slots, budget_bytes=budget, max_iter=args.max_iter,
                              rate_scale=1.0 if rate > 0 else 0.0)
        out = summarize(res, reqs)
        out.update({"rejected": len(rej), "rate_per_s": rate, "peak_bytes_in_use": run_stream.peak_bytes,
                    "peak_running": run_stream.peak_running})
        return out

    common = {"slots": args.slots, "budget_gb": args.budget_gb, "requests": args.requests,
              "precision": "fp16x2 sigma, FP64 Davidson", "max_iter": args.max_iter}
    if args.rate == "auto":
        burst = phase(0.0)
        stream = phase(0.8 * burst["solves_per_s"])
        print(json.dumps(dict(common, burst=burst, poisson_at_80pct=stream)))
    else:
        print(json.dumps(dict(common, **phase(float(args.rate)))))


if __name__ == "__main__":
    main()
