"""The multi-rank logic of bench.py on two CPU ranks (gloo): the step time
is the maximum over ranks, the value counts every replica's work (replica
mode) or the one sigma the ranks share (sub-Hamiltonian split), and the
reference arm prints only on rank 0."""

import json
import os
import socket
import subprocess
import sys

import numpy as np
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    sys.path.insert(0, ROOT)
    import bench
    step = [0.25, 0.75][rank]
    m = bench.world_max(step, dist, "cpu")
    np.save(f"{out}_{rank}.npy", np.array([m, bench.replica_value(1e12, m, world), bench.split_value(1e12, m)]))
    dist.destroy_process_group()


def test_step_time_is_max_over_ranks(tmp_path):
    out = str(tmp_path / "r")
    mp.spawn(_rank, args=(2, _port(), out), nprocs=2, join=True)
    for r in range(2):
        m, v, sv = np.load(f"{out}_{r}.npy")
        assert m == 0.75
        assert abs(v - 2 * 1e12 / 0.75 / 1e12) < 1e-12
        assert abs(sv - 1e12 / 0.75 / 1e12) < 1e-12


def test_reference_arm_other_ranks_print_nothing():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1", "--warmup", "0"],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0 and r.stdout.strip() == ""


def test_reference_arm_line():
    env = dict(os.environ, RANK="0", WORLD_SIZE="1", LOCAL_RANK="0")
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1", "--warmup", "0",
                        "--M", "600"], cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr
    line = json.loads(r.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["cpu_baseline"]["kind"] == "oracle"
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["value"] > 0
