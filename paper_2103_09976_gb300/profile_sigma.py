"""A few sigmas of the middle-bond workload, for a profiler to capture.

K=108 (54|54 spatial orbitals), N=30, 2Sz=0, synthetic N(0,1) operator
blocks (seed 1) over the Gaussian sector dimensions of bond dimension M;
sigma of one seeded normalized psi, `--steps` times, graph replay off so
that every kernel launch is visible to the profiler.

    python -m paper_2103_09976_gb300.profile_sigma --M 800 --prec 3 --steps 3
"""

import argparse

from . import capi


def main():
    import torch
    from synth import gaussian_sector_dims, mirrored_sectors, random_unit_vector
    ap = argparse.ArgumentParser()
    ap.add_argument("--M", type=int, default=800)
    ap.add_argument("--prec", type=int, default=capi.DMRG_FP16X2, help="dmrg_prec: 0 FP64, 1 BF16X2, 2 BF16X3, 3 FP16X2")
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--autotune", action="store_true", help="tune the work split first (as the bench does)")
    ap.add_argument("--producers", type=int, default=0, choices=[0, 1, 3],
                    help="producer warps of the tensor-core kernel (0: the plan's default or the tuner's)")
    args = ap.parse_args()
    left = gaussian_sector_dims(args.M, n_spatial=54, n_tot=30, two_sz_tot=0)
    right = mirrored_sectors(left, n_tot=30, two_sz_tot=0)
    ctx = capi.dmrg_create(device=0, sigma_prec=args.prec, graphs=0, tc_producers=args.producers)
    try:
        capi.dmrg_load_synthetic(ctx, 108, 216, 30, 0, left, right, 1)
        n = capi.dmrg_get_sigma_info(ctx)["psi_size"]
        x = torch.from_numpy(random_unit_vector(n, 1)).cuda()
        y = torch.zeros_like(x)
        if args.autotune:
            capi.dmrg_autotune(ctx, -1)
        for _ in range(args.steps):
            capi.dmrg_sigma(ctx, -1, x, y)
        capi.dmrg_sync(ctx)
        used = capi.dmrg_get_sigma_info(ctx, -1)["tc_producers"]
    finally:
        capi.dmrg_destroy(ctx)
    print("ok", args.M, args.prec, n, "producers", used)


if __name__ == "__main__":
    main()
