"""Precision sweep of the middle-bond sigma at larger bond dimension.

K=108 (54|54 spatial orbitals), N=30, 2Sz=0, synthetic N(0,1) operator
blocks (seed 1), psi ~ N(0,1) normalized: for each M, sigma in FP64 (after
autotuning the FP64 work list) and with the BF16X3 / BF16X2 / FP16X2
tensor-core products, each timed over graph replays with CUDA events on the library's
stream; errors of the mixed results against FP64: max-norm relative error of
sigma and relative error of the Rayleigh quotient psi . sigma.

    python -m paper_2103_09976_gb300.precision_sweep --M 4000 6000
"""

import argparse
import json
import time

import numpy as np

from . import capi

K_ORB, N_EL, TWO_SZ, SEED = 108, 30, 0, 1


def one(M, steps=2, autotune=True, only=None):
    import torch
    from synth import gaussian_sector_dims, mirrored_sectors, random_unit_vector
    left = gaussian_sector_dims(M, n_spatial=K_ORB // 2, n_tot=N_EL, two_sz_tot=TWO_SZ)
    right = mirrored_sectors(left, n_tot=N_EL, two_sz_tot=TWO_SZ)
    ctx = capi.dmrg_create(device=0)
    out = {"M": M}
    try:
        t0 = time.perf_counter()
        capi.dmrg_load_synthetic(ctx, K_ORB, 2 * K_ORB, N_EL, TWO_SZ, left, right, SEED)
        out["load_s"] = time.perf_counter() - t0
        info = capi.dmrg_get_sigma_info(ctx)
        n = info["psi_size"]
        out.update({"psi_size": n, "flops": info["flops"], "op_elements": info["op_elements"]})
        x = torch.from_numpy(random_unit_vector(n, SEED)).cuda()
        stream = torch.cuda.ExternalStream(capi.dmrg_stream(ctx))
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ref = None
        for name, prec in (("fp64", capi.DMRG_FP64), ("bf16x3", capi.DMRG_BF16X3), ("bf16x2", capi.DMRG_BF16X2),
                           ("fp16x2", capi.DMRG_FP16X2)):
            if only and name != "fp64" and name not in only:
                continue
            capi.dmrg_set_precision(ctx, prec)
            t0 = time.perf_counter()
            if prec == capi.DMRG_FP64 and autotune:
                out["autotuned"] = capi.dmrg_autotune(ctx, -1)
            y = torch.zeros(n, dtype=torch.float64, device="cuda")
            tuned = None
            try:
                for _ in range(2):
                    capi.dmrg_sigma(ctx, -1, x, y)
                capi.dmrg_sync(ctx)
                if prec != capi.DMRG_FP64:   # tensor-core work split, picked by timing
                    tuned = capi.dmrg_autotune(ctx, -1)
                    capi.dmrg_sigma(ctx, -1, x, y)
                    capi.dmrg_sync(ctx)
            except capi.DMRGError as ex:   # e.g. the split slices do not fit next to the FP64 store
                out[name] = {"error": str(ex)}
                continue
            prep = time.perf_counter() - t0
            e0.record(stream)
            for _ in range(steps):
                capi.dmrg_sigma(ctx, -1, x, y)
            e1.record(stream)
            e1.synchronize()
            s = e0.elapsed_time(e1) / 1e3 / steps
            r = {"ms": s * 1e3, "tflops": info["flops"] / s / 1e12, "prep_s": prep}
            if tuned is not None:
                nprod = 6 if prec == capi.DMRG_BF16X3 else 3
                # operators once as 3 bf16 slices (2 fp16 slices for FP16X2), psi, sigma
                alg = (4.0 if prec == capi.DMRG_FP16X2 else 6.0) * info["op_elements"] + 16.0 * n
                r.update({"tc_items_per_sm": tuned[0], "tc_unit_cost": tuned[1],
                          "tc_producers": capi.dmrg_get_sigma_info(ctx, -1)["tc_producers"], "hbm_gbs": alg / s / 1e9,
                          "tensor_tflops_issued": nprod * info["flops"] / s / 1e12})
            if ref is None:
                ref = y.clone()
            else:
                r["rel_err_maxnorm"] = (y - ref).abs().max().item() / ref.abs().max().item()
                r["rayleigh_rel_err"] = abs(float(x @ y) - float(x @ ref)) / abs(float(x @ ref))
            out[name] = r
    finally:
        capi.dmrg_destroy(ctx)
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--M", type=int, nargs="+", default=[4000, 6000])
    ap.add_argument("--steps", type=int, default=2)
    ap.add_argument("--no-autotune", action="store_true")
    ap.add_argument("--only", nargs="+", default=None, choices=["bf16x3", "bf16x2", "fp16x2"],
                    help="mixed precisions to run (FP64, the reference, always runs)")
    args = ap.parse_args()
    for M in args.M:
        print(json.dumps(one(M, args.steps, not args.no_autotune, args.only)), flush=True)


if __name__ == "__main__":
    main()
