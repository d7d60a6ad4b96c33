"""Energy error of the mixed-precision sigma on one fixed effective Hamiltonian.

Sweep energies of two precisions drift apart through their different
truncation paths, so they do not isolate the sigma's precision. Here the
blocks are built from seeded integrals (FeMoco-shaped by default: K
orbitals, N = round(113 K / 76) electrons, 2Sz = N mod 2, mixed NC/CN cut in
the middle) and carried through one forward sweep at bond dimension M (BF16X3
sigma, |r|^2 <= 1e-6), which fixes the middle bond's H_eff; its lowest
eigenvalue is then solved with each sigma precision: FP64 to |r|^2 <=
1e-10, the mixed precisions to |r|^2 <= tol_mixed. Every
reported eigenvalue is the FP64 Rayleigh quotient of the solver's vector, so
the differences are the energy error the mixed sigma leaves after a solve.

    python -m paper_2103_09976_gb300.bond_energy --K 76 --M 500 1000
"""

import argparse
import json
import time

from . import capi


def one(K, M, seed=2, tol_mixed=1e-7, max_iter=400, precs=("BF16X3", "FP16X2", "BF16X2")):
    from synth.integrals import femoco_like_integrals
    N = 113 * K // 76
    two_sz = N % 2
    t, v = femoco_like_integrals(K=K, seed=seed)
    ctx = capi.dmrg_create(device=0, seed=seed, dav_max_iter=max_iter, mixed_cut=K // 2)
    out = {"K": K, "N": N, "two_sz": two_sz, "M": M, "site": K // 2 - 1, "integrals": "femoco-shaped", "seed": seed}
    try:
        capi.dmrg_build_blocks(ctx, t, v, K, N, two_sz, M)
        capi.dmrg_set_precision(ctx, capi.DMRG_BF16X3)
        t0 = time.perf_counter()
        capi.dmrg_sweep(ctx, [M], 1e-6)
        out["sweep_s"] = time.perf_counter() - t0
        site = K // 2 - 1
        n = capi.dmrg_psi_layout(ctx, site)["size"]
        out["psi_size"] = n
        ref = None
        for name in ("FP64",) + tuple(precs):
            capi.dmrg_set_precision(ctx, getattr(capi, "DMRG_" + name))
            t0 = time.perf_counter()
            e, it, conv = capi.dmrg_davidson(ctx, site, None, 1e-10 if name == "FP64" else tol_mixed)
            r = {"energy": e, "products": it, "converged": conv, "s": time.perf_counter() - t0}
            if ref is None:
                ref = e
            else:
                r["error_vs_fp64"] = e - ref
            out[name.lower()] = r
    finally:
        capi.dmrg_destroy(ctx)
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--K", type=int, default=76)
    ap.add_argument("--M", type=int, nargs="+", default=[500])
    ap.add_argument("--seed", type=int, default=2)
    ap.add_argument("--tol-mixed", type=float, default=1e-7)
    args = ap.parse_args()
    for M in args.M:
        print(json.dumps(one(args.K, M, args.seed, args.tol_mixed)), flush=True)


if __name__ == "__main__":
    main()
