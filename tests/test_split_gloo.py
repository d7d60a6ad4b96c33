"""Two CPU ranks (gloo) each compute their sub-Hamiltonian part of sigma
with the oracle and sum them with one all-reduce, the only exchange of the
split (Sec. II.B); the result equals the full sigma."""

import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _problem(cn=False):
    if cn:  # a CN bond (Eq. h-cn) over exact Fock-space blocks: K=4, cut after 2 orbitals
        from oracle.cn import cn_terms
        from oracle.nc import Integrals, fock_ops_exact
        from oracle.sigma import psi_layout
        from synth import random_integrals, random_unit_vector
        t, v = random_integrals(4, 6)
        ints = Integrals(t, v)
        bL, _, oL = fock_ops_exact(ints, list(range(4)), "L", "cn")
        bR, _, oR = fock_ops_exact(ints, list(range(4, 8)), "R", "cn")
        lay, size = psi_layout(bL, bR, (4, 0))
        return lay, cn_terms(4, 8), oL, oR, random_unit_vector(size, 5)
    from oracle.nc import nc_terms
    from oracle.sigma import psi_layout, synthetic_ops
    from synth import gaussian_sector_dims, mirrored_sectors, random_unit_vector
    left = gaussian_sector_dims(40, n_spatial=3, n_tot=6)
    right = mirrored_sectors(left, n_tot=6)
    bL, bR, oL, oR, _ = synthetic_ops(left, right, 6, 12, seed=2)
    lay, size = psi_layout(bL, bR, (6, 0))
    return lay, nc_terms(6, 12), oL, oR, random_unit_vector(size, 3)


def _rank_main(rank, world, port, out_path, cn=False):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from oracle.sigma import sigma_part
    lay, terms, oL, oR, x = _problem(cn)
    part = torch.from_numpy(sigma_part(x, lay, terms, oL, oR, rank, world))
    dist.all_reduce(part, op=dist.ReduceOp.SUM)
    if rank == 0:
        np.save(out_path, part.numpy())
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("cn", [False, True])
def test_allreduce_of_parts_is_full_sigma(tmp_path, cn):
    """NC terms (Eq. proc-def-nc) and CN terms (Eq. proc-def-cn)."""
    from oracle.sigma import sigma_blocks
    out = str(tmp_path / "sigma.npy")
    mp.spawn(_rank_main, args=(2, _free_port(), out, cn), nprocs=2, join=True)
    lay, terms, oL, oR, x = _problem(cn)
    full = sigma_blocks(x, lay, terms, oL, oR)
    got = np.load(out)
    assert np.abs(got - full).max() <= 1e-13 * np.abs(full).max()
