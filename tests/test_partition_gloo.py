"""The library's partition of the middle-bond problem into sub-Hamiltonians
(Sec. II.B, Eqs. sum-h, sub-h, proc-def, proc-def-nc), as the multi-GPU
sigma uses it, driven from two CPU ranks (gloo) through the host-only C ABI
call dmrg_partition_info (no GPU needed): each rank asks the library which
terms it owns and how many operator elements it stores; the ranks exchange
their answers with collectives. The term sets are disjoint, their union is
every NC term, each term's owner is the oracle's rank for it
(oracle.sigma.nc_term_rank), and the stored operator elements of all ranks
add up to the full store, each rank holding about 1/world of it."""

import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

CASES = {  # (spin orbitals left, total, N, 2Sz, M per side, spatial orbitals per side)
    "small": (8, 16, 8, 0, 60, 4),
    "k108_m2000": (108, 216, 30, 0, 2000, 54),
}


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _sectors(case):
    from synth import gaussian_sector_dims, mirrored_sectors
    nL, n, N, tsz, M, nsp = CASES[case]
    left = gaussian_sector_dims(M, n_spatial=nsp, n_tot=N, two_sz_tot=tsz)
    return left, mirrored_sectors(left, n_tot=N, two_sz_tot=tsz)


def _rank_main(rank, world, port, case, out_dir):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from paper_2103_09976_gb300 import capi
    nL, n, N, tsz, M, nsp = CASES[case]
    left, right = _sectors(case)
    info = capi.dmrg_partition_info(nL, n, N, tsz, left, right, rank, world, max_ids=1 << 20)
    ids = torch.from_numpy(np.asarray(info["term_ids"], dtype=np.int64))
    counts = [torch.zeros(1, dtype=torch.int64) for _ in range(world)]
    dist.all_gather(counts, torch.tensor([len(ids)], dtype=torch.int64))
    width = int(max(c.item() for c in counts))
    padded = torch.full((width,), -1, dtype=torch.int64)
    padded[:len(ids)] = ids
    gathered = [torch.zeros(width, dtype=torch.int64) for _ in range(world)]
    dist.all_gather(gathered, padded)
    elems = torch.tensor([info["op_elements"]], dtype=torch.int64)
    total_elems = elems.clone()
    dist.all_reduce(total_elems, op=dist.ReduceOp.SUM)
    if rank == 0:
        np.savez(os.path.join(out_dir, "part.npz"),
                 ids=np.stack([g.numpy() for g in gathered]),
                 counts=np.array([c.item() for c in counts]),
                 elems_sum=total_elems.item(), total=info["total_elements"])
    np.save(os.path.join(out_dir, f"elems{rank}.npy"), np.array([info["op_elements"], info["n_terms"]]))
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("case", list(CASES))
def test_partition_covers_every_term_once(tmp_path, case):
    pytest.importorskip("ctypes")
    from oracle.nc import nc_terms
    from oracle.sigma import nc_term_rank
    from paper_2103_09976_gb300 import build, capi
    if not os.path.exists(capi.LIB_PATH):
        build.build()
    world = 2
    mp.spawn(_rank_main, args=(world, _free_port(), case, str(tmp_path)), nprocs=world, join=True)
    d = np.load(tmp_path / "part.npz")
    nL, n = CASES[case][0], CASES[case][1]
    terms = nc_terms(nL, n)
    owner = np.full(len(terms), -1)
    for r in range(world):
        got = d["ids"][r][:d["counts"][r]]
        assert np.all(owner[got] == -1), "a term is owned by two ranks"
        owner[got] = r
    assert np.all(owner >= 0), "a term is owned by no rank"
    assert owner.tolist() == [nc_term_rank(t, world) for t in terms]
    assert int(d["elems_sum"]) == int(d["total"])
    for r in range(world):
        e, nt = np.load(tmp_path / f"elems{r}.npy")
        assert abs(e / d["total"] - 1.0 / world) < 0.1, (r, e, d["total"])
