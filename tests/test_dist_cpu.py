"""Multi-rank host logic of the benchmark on CPU `gloo` ranks (world size 2): every rank gets its
own molecule, the timed duration is the maximum over ranks and the throughput counts all ranks'
pair*q; each rank's profile (here from the CPU oracle, standing in for its GPU) is its own."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    import torch.distributed as dist

    import bench
    import oracle
    from paper_1306_2258_gb300 import workloads as wl
    dist.init_process_group("gloo", rank=rank, world_size=world)
    mol = bench.rank_molecule(None, rank, n=300)
    coef = wl.form_factor_coefficients(5, wl.seed_for(2, 1))
    q = wl.q_grid(0.0, 1.0, 21)
    I = oracle.profile(mol.coords, mol.types, coef, q)
    pq = mol.n * (mol.n - 1) // 2 * q.size
    tot_ms = 100.0 * (rank + 1)                  # rank 1 is the slow one
    max_ms, value = bench.aggregate(tot_ms, pq, 4, world)
    out[rank] = (max_ms, value, float(I[3]), pq)
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_weak_scaling_aggregation():
    world = 2
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_worker, args=(world, _free_port(), out), nprocs=world, start_method="spawn", join=True)
    (m0, v0, i0, pq0), (m1, v1, i1, pq1) = out[0], out[1]
    assert m0 == m1 == 200.0
    assert v0 == v1 == pytest.approx((pq0 + pq1) * 4 / 0.2)
    assert i0 != i1                                 # independent problems
