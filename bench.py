"""Benchmark: sigma = H_eff . psi at the middle bond of two-site ab initio DMRG.

Workload (default): K=108 spatial orbitals split 54|54, N=30, 2Sz=0, bond
dimension M=2000 per side (104 sectors, |psi| = 106,004), 23,654 NC terms,
synthetic N(0,1) operator blocks (seed 1), FP64 arithmetic. One step = one
sigma call with psi and the operators resident in HBM.

Prints one JSON line (rank 0). Roofline of the FP64 kernel: algorithmic
FLOPs per launch (sum over terms and blocks of the cheaper contraction
order) over its CUDA-event duration, against cuBLAS DGEMM measured in the
same run; mixed precision: algorithmic bytes (every stored operator element
once as three bf16 slices, psi, sigma) over the kernel duration, against the
measured HBM bandwidth.
  python bench.py [--gpus N] [--steps K] [--warmup W] [--M 2000] [--impl ours|reference] [--replicas]

With N > 1 ranks (torchrun, one GPU each) the sigma is split by the paper's
sub-Hamiltonian partition (Sec. II.B): every rank stores only the operators
of its sub-Hamiltonian (dmrg_load_synthetic_part, about 1/N of the store),
computes its part of sigma, and one NCCL all-reduce of |psi| doubles per
step sums the parts (strong scaling: the job does one full sigma per step).
--replicas instead runs N independent full problems (weak scaling).
"""

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

K_ORB, N_EL, TWO_SZ, SEED = 108, 30, 0, 1
METRIC = "H_eff.psi TFLOP/s (middle-bond sigma)"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--M", type=int, default=2000)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--e2e-steps", type=int, default=3)
    ap.add_argument("--no-serve", action="store_true")
    ap.add_argument("--serve-requests", type=int, default=32)
    ap.add_argument("--no-sweeps", action="store_true")
    ap.add_argument("--replicas", action="store_true",
                    help="N>1: N independent full problems instead of the sub-Hamiltonian split")
    return ap.parse_args()


def workload(M):
    from synth import gaussian_sector_dims, mirrored_sectors
    left = gaussian_sector_dims(M, n_spatial=K_ORB // 2, n_tot=N_EL, two_sz_tot=TWO_SZ)
    right = mirrored_sectors(left, n_tot=N_EL, two_sz_tot=TWO_SZ)
    return left, right


def config(M, prec="fp64"):
    return {"workload": f"middle-bond sigma, K={K_ORB} (54|54 spatial orbitals), N={N_EL}, 2Sz={TWO_SZ}, "
                        f"M={M}, 23654 NC terms, synthetic N(0,1) operator blocks seed {SEED}",
            "K": K_ORB, "N": N_EL, "two_sz": TWO_SZ, "M": M, "sigma_precision": prec,
            "l2": "inputs larger than L2 (operator store >> 129 MB), no flush"}


# DRAM bytes per sigma at M=2000, from ncu captures of the small case M=800
# scaled by the bytes each kernel requests (counted with the kernels' own
# formulas by tests/host/plan_check.cpp) at both sizes:
# profiles/sigma_f64_middle_bond_m800_dram.md, sigma_mixed_middle_bond_m800_dram.md.
F64_TRAFFIC_M2000 = 70.0e9
MIXED_TRAFFIC_M2000 = {"bf16x3": 32.4e9, "bf16x2": 32.4e9, "fp16x2": 20.6e9}
TRAFFIC_SOURCE = ("ncu dram__bytes_read.sum + dram__bytes_write.sum at M=800 (small case) per requested byte, "
                  "times the requested bytes at M=2000")

# ------------------------------------------------------------------ clocks
class Clocks:
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.p = None

    def start(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.p.terminate()
        self.p.wait()
        self.f.seek(0)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.f.read().splitlines():
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        os.unlink(self.f.name)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------------- oracle leg
def oracle_sample(M, n_terms):
    """The oracle's sigma on the first n_terms NC terms of the workload (a
    bounded sample of the same middle-bond problem). Returns (run, flops)."""
    from oracle.nc import nc_terms
    from oracle.sigma import psi_layout, sigma_blocks, sigma_flops, synthetic_op_specs, synthetic_ops
    from synth import random_unit_vector
    left, right = workload(M)
    terms = nc_terms(K_ORB, 2 * K_ORB)[:n_terms]
    need = set()
    for kl, tl, kr, tr, c in terms:
        if kl is not None:
            need.add(("L", kl))
        if kr is not None:
            need.add(("R", kr))
    bL, bR, oL, oR, _ = synthetic_ops(left, right, K_ORB, 2 * K_ORB, SEED, only=need)
    lay, size = psi_layout(bL, bR, (N_EL, TWO_SZ))
    specs = synthetic_op_specs(K_ORB, 2 * K_ORB)
    dqL = {k: dq for s, k, dq, _ in specs if s == "L"}
    dqR = {k: dq for s, k, dq, _ in specs if s == "R"}
    flops = sigma_flops(lay, terms, dqL, dqR, bL, bR)
    x = random_unit_vector(size, SEED)

    def run():
        return sigma_blocks(x, lay, terms, oL, oR)
    return run, flops


def cpu_baseline(M, n_terms=700, reps=12):
    run, flops = oracle_sample(M, n_terms)
    t0 = time.perf_counter()
    for _ in range(reps):
        run()
    dt = (time.perf_counter() - t0) / reps
    return {"value": flops / dt / 1e12, "unit": "TFLOP/s", "cores": os.cpu_count(), "kind": "oracle",
            "sample": f"oracle sigma (numpy FP64, per-term per-block loop), {reps} repetitions over the first {n_terms} of "
                      f"23654 NC terms at M={M}: {flops / 1e9:.1f} GFLOP in {dt:.2f} s per repetition "
                      f"({reps * dt:.1f} s of CPU work in all)"}


def run_reference(args, rank):
    if rank != 0:
        return
    n_terms = 700
    run, flops = oracle_sample(args.M, n_terms)
    for _ in range(args.warmup):
        run()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        run()
    dt = (time.perf_counter() - t0) / args.steps
    v = flops / dt / 1e12
    out = {"metric": METRIC, "value": v, "unit": "TFLOP/s", "n_gpus": args.gpus, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": dt * 1e3, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
           "config": config(args.M),
           "cpu_baseline": {"value": v, "unit": "TFLOP/s", "cores": os.cpu_count(), "kind": "oracle",
                            "sample": f"first {n_terms} of 23654 NC terms per step, {flops / 1e9:.1f} GFLOP"},
           "e2e": {"value": v, "unit": "TFLOP/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


# ---------------------------------------------------------------- our leg
def fp64_gemm_peak(torch):
    n = 4096
    a = torch.randn(n, n, dtype=torch.float64, device="cuda")
    b = torch.randn(n, n, dtype=torch.float64, device="cuda")
    for _ in range(2):
        torch.matmul(a, b)
    torch.cuda.synchronize()
    best = 1e9
    for _ in range(5):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        torch.matmul(a, b)
        e1.record()
        e1.synchronize()
        best = min(best, e0.elapsed_time(e1) / 1e3)
    return 2.0 * n ** 3 / best / 1e12


def world_max(x, dist, device):
    """Largest value of x over all ranks (the job's step time is the slowest rank's)."""
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_value(flops_per_step, step_s, world):
    """Whole-job throughput of `world` replicas that each run one problem per step."""
    return world * flops_per_step / step_s / 1e12


def split_value(flops_full, step_s):
    """Whole-job throughput of the sub-Hamiltonian split: one full sigma per
    step, its work divided among the ranks; step_s is the slowest rank's."""
    return flops_full / step_s / 1e12


def serve_section(n_req, device):
    """Davidson solves through the native serving loop: first a burst (all
    requests at t=0) to measure capacity, then a Poisson stream at 80% of it."""
    from paper_2103_09976_gb300 import serve
    from synth.requests import poisson_requests
    kw = dict(k_choices=(24, 36, 54), m_choices=(250, 500, 1000))
    reqs = poisson_requests(n_req, rate_per_s=1.0, seed=5, **kw)
    res, rej = serve.run_stream(reqs, n_slots=4, device=device, rate_scale=0.0)
    burst = serve.summarize(res, reqs)
    rate = 0.8 * burst["solves_per_s"]
    reqs = poisson_requests(n_req, rate_per_s=rate, seed=6, **kw)
    res, rej2 = serve.run_stream(reqs, n_slots=4, device=device, rate_scale=1.0)
    stream = serve.summarize(res, reqs)
    return {"workload": f"{n_req} Davidson solves per run, middle-bond problems K in {{24,36,54}}, "
                        "M in {250,500,1000}, N ~ U[K/2,K], synthetic operators seeded per request; "
                        "fp16x2 sigma, FP64 Davidson, tol 1e-8, at most 60 sigma calls; 4 slots, 160 GB budget",
            "burst": {k: burst[k] for k in ("p50_s", "p99_s", "solves_per_s", "ok")},
            "poisson_at_80pct": {k: stream[k] for k in ("p50_s", "p99_s", "solves_per_s", "ok")},
            "rate_per_s": rate, "rejected": len(rej) + len(rej2)}


def sweeps_section(device):
    """Two sweeps of a FeMoco-shaped problem with the NC partition everywhere
    and with the mixed NC/CN partition (Sec. III.A): wall time (initial blocks
    included), energies, converged steps."""
    from paper_2103_09976_gb300 import sweeps
    out = {"workload": "K=36 spatial orbitals, N=53, 2Sz=1, FeMoco-shaped integrals (seed 2), M 250 then 250; "
                       "fp16x2 sigma, FP64 Davidson (tol 1e-6, at most 60 products, carried start vectors), "
                       "FP64 decimation and transformation; mixed cut after 18 orbitals"}
    for name, cut in (("nc", -1), ("mixed_nc_cn", 18)):
        r = sweeps.run(36, [250, 250], cut, "FP16X2", device=device)
        out[name] = {"s": r["build_s"] + r["sweeps_s"], "energies": r["energies"], "converged": r["converged"],
                     "steps": r["steps"], "phase_s": r["phase_s"]}
    out["nc_over_mixed"] = out["nc"]["s"] / out["mixed_nc_cn"]["s"]
    return out


def main():
    args = parse()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank)
        return
    import numpy as np
    import torch
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    from paper_2103_09976_gb300 import capi
    from synth import random_unit_vector

    left, right = workload(args.M)
    split = world > 1 and not args.replicas
    ctx = capi.dmrg_create(device=local)
    if split:   # this rank's sub-Hamiltonian: its terms and only the operators they use
        capi.dmrg_load_synthetic_part(ctx, K_ORB, 2 * K_ORB, N_EL, TWO_SZ, left, right, SEED, rank, world)
    else:
        capi.dmrg_load_synthetic(ctx, K_ORB, 2 * K_ORB, N_EL, TWO_SZ, left, right, SEED)
    info = capi.dmrg_get_sigma_info(ctx)
    n = info["psi_size"]
    x_h = random_unit_vector(n, SEED)
    x = torch.from_numpy(x_h).cuda()
    y = torch.zeros(n, dtype=torch.float64, device="cuda")
    stream = torch.cuda.ExternalStream(capi.dmrg_stream(ctx))
    flops_full = info["flops"]
    if split:   # the job's work per step: all ranks' parts of one sigma
        t = torch.tensor([info["flops"]], dtype=torch.float64, device="cuda")
        dist.all_reduce(t)
        flops_full = float(t.item())

    def step(xin, yout):
        """One sigma of the job: this rank's part, then (split) the sum over ranks."""
        capi.dmrg_sigma(ctx, -1, xin, yout)
        if split:
            with torch.cuda.stream(stream):
                dist.all_reduce(yout)

    tuned = capi.dmrg_autotune(ctx, -1)   # work-list split and order of the FP64 kernel
    for _ in range(max(3, args.warmup)):
        step(x, y)
    torch.cuda.synchronize()
    clk = Clocks(local)
    clk.start()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    # timed steps: each sigma is one replay of its captured graph
    e0.record(stream)
    for _ in range(args.steps):
        step(x, y)
    e1.record(stream)
    e1.synchronize()
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    step_s = e0.elapsed_time(e1) / 1e3 / args.steps
    # kernel durations for the roofline: the same steps launched directly
    # with CUDA events around each kernel on the library's stream
    capi.dmrg_profile(ctx, True)
    for _ in range(args.steps):
        capi.dmrg_sigma(ctx, -1, x, y)
    k_ms, k_n = capi.dmrg_profile_read(ctx, capi.KERNEL_SIGMA)
    r_ms, r_n = capi.dmrg_profile_read(ctx, capi.KERNEL_REDUCE)
    capi.dmrg_profile(ctx, False)
    clocks = clk.stop()
    if dist:
        step_s = world_max(step_s, dist, "cuda")

    # end to end with pinned host buffers: psi in, sigma out every step
    xp = torch.from_numpy(x_h).pin_memory()
    yp = torch.zeros(n, dtype=torch.float64).pin_memory()

    def e2e_step():
        if not split:   # the C ABI stages host buffers itself
            capi.dmrg_sigma(ctx, -1, xp, yp)
            return
        with torch.cuda.stream(stream):
            xd = xp.to("cuda", non_blocking=True)
            yd = torch.empty_like(xd)
        step(xd, yd)
        with torch.cuda.stream(stream):
            yp.copy_(yd, non_blocking=True)
        stream.synchronize()

    e2e_step()
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    t0 = time.perf_counter()
    for _ in range(args.e2e_steps):
        e2e_step()
    e2e_s = (time.perf_counter() - t0) / args.e2e_steps
    if dist:
        e2e_s = world_max(e2e_s, dist, "cuda")
    ok = bool(np.allclose(yp.numpy(), y.cpu().numpy(), rtol=0, atol=1e-12 * float(y.abs().max())))

    # tensor-core sigma (bf16 slices) on the same context and psi
    flops = info["flops"]
    mixed = {}
    mixed_precisions = () if split else (("bf16x3", capi.DMRG_BF16X3, 6, 6), ("bf16x2", capi.DMRG_BF16X2, 3, 6),
                                         ("fp16x2", capi.DMRG_FP16X2, 3, 4))
    y64 = y.clone()
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        peaks = {}
    hbm = float(peaks.get("hbm_gbs", 6800.0))
    bf16 = float(peaks.get("bf16_tflops", 1900.0))
    for name, prec, nprod, bytes_per_elem in mixed_precisions:
        capi.dmrg_set_precision(ctx, prec)
        capi.dmrg_sigma(ctx, -1, x, y)  # builds the operator slices of this precision
        capi.dmrg_sync(ctx)
        tc_tuned = capi.dmrg_autotune(ctx, -1)  # items per SM, unit cost and producer warps of the tensor-core path
        tc_producers = capi.dmrg_get_sigma_info(ctx, -1)["tc_producers"]
        for _ in range(max(3, args.warmup)):
            capi.dmrg_sigma(ctx, -1, x, y)
        capi.dmrg_sync(ctx)
        e0.record(stream)
        for _ in range(args.steps):
            capi.dmrg_sigma(ctx, -1, x, y)
        e1.record(stream)
        e1.synchronize()
        capi.dmrg_sync(ctx)
        step = e0.elapsed_time(e1) / 1e3 / args.steps
        capi.dmrg_profile(ctx, True)          # kernel durations, launched directly
        for _ in range(args.steps):
            capi.dmrg_sigma(ctx, -1, x, y)
        capi.dmrg_sync(ctx)
        tms, tn = capi.dmrg_profile_read(ctx, capi.KERNEL_SIGMA)
        capi.dmrg_profile(ctx, False)
        kern = tms / 1e3 / max(1, tn)
        d = (y - y64).abs().max().item() / y64.abs().max().item()
        rq = abs(float(x @ y) - float(x @ y64)) / abs(float(x @ y64))
        # algorithmic bytes: every stored operator element once (6 B as three
        # bf16 slices, 4 B as two fp16 slices) + psi read + sigma written (FP64)
        alg_bytes = info["op_elements"] * bytes_per_elem + 16.0 * n
        traffic = MIXED_TRAFFIC_M2000[name] if args.M == 2000 else None
        mixed[name] = {"value": flops / step / 1e12, "unit": "TFLOP/s", "ms_per_step": step * 1e3,
                       "kernel_ms": kern * 1e3, "rel_err_vs_fp64_maxnorm": d, "rayleigh_rel_err_vs_fp64": rq,
                       "speedup_vs_fp64_kernel": (k_ms / max(1, k_n)) / (kern * 1e3),
                       "autotuned": {"tc_items_per_sm": tc_tuned[0], "tc_unit_cost": tc_tuned[1],
                                     "tc_producers": tc_producers, "tune_ms": tc_tuned[2]},
                       "roofline": {"bound": "hbm", "achieved": alg_bytes / kern / 1e9, "peak": hbm,
                                    "unit": "GB/s", "frac": alg_bytes / kern / 1e9 / hbm, "traffic": traffic,
                                    "traffic_source": TRAFFIC_SOURCE if traffic else None,
                                    "kernel": "sigma_small_kernel + sigma_tc_kernel (one sigma)",
                                    "peak_source": "MEASURED_PEAKS.json hbm_gbs",
                                    "tensor_tflops_issued": nprod * flops / kern / 1e12,
                                    "tensor_frac_of_bf16_peak": nprod * flops / kern / 1e12 / bf16}}
    capi.dmrg_set_precision(ctx, capi.DMRG_FP64)
    peak64 = fp64_gemm_peak(torch)
    capi.dmrg_destroy(ctx)
    serving = None if (args.no_serve or world > 1) else serve_section(args.serve_requests, local)

    kern_s = k_ms / 1e3 / max(1, k_n)
    achieved = flops / kern_s / 1e12
    value = split_value(flops_full, step_s) if split else replica_value(flops, step_s, world)
    out = {"metric": METRIC, "value": value, "unit": "TFLOP/s", "n_gpus": world, "steps": args.steps,
           "warmup": max(3, args.warmup), "ms_per_step": step_s * 1e3, "higher_is_better": True,
           "scaling": "strong" if split else "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": dict(config(args.M), parallelism=(f"sub-Hamiltonian split over {world} ranks, NCCL all-reduce "
                                                       "of sigma" if split else
                                                       (f"{world} replicas" if world > 1 else "1 GPU"))),
           "roofline": {"bound": "alu", "achieved": achieved, "peak": peak64, "unit": "TFLOP/s",
                        "frac": achieved / peak64,
                        "traffic": F64_TRAFFIC_M2000 if args.M == 2000 else None,
                        "traffic_source": TRAFFIC_SOURCE + " (profiles/sigma_f64_middle_bond_m800_dram.md)",
                        "kernel": "sigma_f64_kernel",
                        "peak_source": "cuBLAS DGEMM 4096^3 measured in this run (no FP64 entry in MEASURED_PEAKS.json); "
                                       "cross-check: measured bf16 x nominal FP64/bf16 ratio = "
                                       f"{bf16 * 1.25 / 2250.0:.3f} TFLOP/s",
                        "kernel_ms": kern_s * 1e3, "reduce_ms": r_ms / max(1, r_n),
                        "autotuned": {"items_per_sm": tuned[0], "per_task_cost": tuned[1], "tune_ms": tuned[2]}},
           "e2e": {"value": (flops_full if split else world * flops) / e2e_s / 1e12, "unit": "TFLOP/s",
                   "h2d_bytes_per_step": 8 * n,
                   "d2h_bytes_per_step": 8 * n, "matches_device_result": ok},
           "gpu_launches": 2 * args.steps,
           "mixed": mixed,
           "serving": serving,
           "clocks": clocks,
           "sigma_info": info}
    if rank == 0 and world == 1 and not args.no_sweeps:
        try:
            out["sweeps"] = sweeps_section(local)
        except Exception as ex:  # reported, not fatal: the headline above is complete
            out["sweeps"] = {"error": str(ex)[:300]}
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(args.M)
    if rank == 0:
        print(json.dumps(out), flush=True)
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
