"""Two-site DMRG sweeps from seeded synthetic integrals, timed per phase.

Random real integrals (t symmetric N(0,1), v 8-fold symmetric N(0, 0.1^2)),
optionally with the FeMoco-shaped decay exp(-(|i-j| + |k-l|)/8); N defaults
to the FeMoco filling round(113 K / 76) and 2Sz to N mod 2. One JSON line per
partition with sweep energies, discarded weights, wall time per sweep and
per phase (blocking, Davidson, decimation, transformation), Davidson
products and convergence, and the per-site time of the last sweep.

    python -m paper_2103_09976_gb300.sweeps --K 76 --M 250,500 --cut -1 38
"""

import argparse
import json
import time

from . import capi


def run(K, schedule, cut, prec="FP16X2", N=None, two_sz=None, seed=2, femoco=True, tol=1e-6, max_iter=60,
        noise=0.0, device=0):
    from synth.integrals import femoco_like_integrals, random_integrals
    N = 113 * K // 76 if N is None else N
    two_sz = N % 2 if two_sz is None else two_sz
    t, v = femoco_like_integrals(K=K, seed=seed) if femoco else random_integrals(K, seed)
    ctx = capi.dmrg_create(device=device, seed=seed, dav_max_iter=max_iter, noise=noise,
                           sigma_prec=getattr(capi, "DMRG_" + prec), mixed_cut=cut)
    try:
        t0 = time.perf_counter()
        capi.dmrg_build_blocks(ctx, t, v, K, N, two_sz, schedule[0])
        t1 = time.perf_counter()
        e, d = capi.dmrg_sweep(ctx, schedule, tol)
        t2 = time.perf_counter()
        log = capi.dmrg_sweep_log(ctx)
    finally:
        capi.dmrg_destroy(ctx)
    phases = ("t_block", "t_solve", "t_decimate", "t_transform")
    last = len(schedule) - 1
    return {"K": K, "N": N, "two_sz": two_sz, "cut": cut, "prec": prec, "schedule": list(schedule),
            "integrals": "femoco-shaped" if femoco else "random", "seed": seed,
            "build_s": t1 - t0, "sweeps_s": t2 - t1, "energies": [float(x) for x in e],
            "max_discarded": [float(x) for x in d],
            "per_sweep_s": [sum(l[k] for l in log if l["sweep"] == s for k in phases) for s in range(len(schedule))],
            "phase_s": {k: sum(l[k] for l in log) for k in phases},
            "products": sum(l["iters"] for l in log), "steps": len(log),
            "converged": sum(l["converged"] for l in log),
            "max_kept": max(l["kept"] for l in log), "max_psi": max(l["psi_size"] for l in log),
            "last_sweep_site_s": {l["site"]: round(sum(l[k] for k in phases), 4) for l in log if l["sweep"] == last}}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--K", type=int, default=24)
    ap.add_argument("--M", default="80,80", help="bond dimension per sweep (forward, backward, ...)")
    ap.add_argument("--cut", type=int, nargs="+", default=[-1], help="mixed NC/CN cut(s); -1 = NC everywhere")
    ap.add_argument("--prec", default="FP16X2", choices=["FP64", "BF16X3", "BF16X2", "FP16X2"])
    ap.add_argument("--N", type=int, default=None)
    ap.add_argument("--two-sz", type=int, default=None)
    ap.add_argument("--seed", type=int, default=2)
    ap.add_argument("--random", action="store_true", help="undecayed random integrals")
    ap.add_argument("--tol", type=float, default=1e-6)
    ap.add_argument("--max-iter", type=int, default=60)
    ap.add_argument("--noise", type=float, default=0.0)
    args = ap.parse_args()
    sched = [int(x) for x in args.M.split(",")]
    for cut in args.cut:
        print(json.dumps(run(args.K, sched, cut, args.prec, args.N, args.two_sz, args.seed, not args.random,
                             args.tol, args.max_iter, args.noise)), flush=True)


if __name__ == "__main__":
    main()
