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


def _share_worker(rank, world, port, out, fail_rank):
    """Rank r computes the oracle's share of the rows i in its block (I of the suffix from the
    block's start minus I of the suffix after it), then the shares are combined over gloo."""
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    import datetime

    import torch
    import torch.distributed as dist

    import oracle
    from paper_1306_2258_gb300 import workloads as wl
    from paper_1306_2258_gb300.shard import allreduce_shares
    dist.init_process_group("gloo", rank=rank, world_size=world, timeout=datetime.timedelta(seconds=5))
    mol = wl.random_walk_globule(240, 4, 77)
    coef = wl.form_factor_coefficients(4, 78)
    q = wl.q_grid(0.0, 0.8, 33)
    n = mol.n
    s, e = rank * n // world, (rank + 1) * n // world

    def suffix(k):
        return oracle.profile(mol.coords[k:], mol.types[k:], coef, q) if k < n else np.zeros(q.size)

    share = torch.as_tensor(suffix(s) - suffix(e))
    if rank == fail_rank:   # this rank leaves before the collective
        out[rank] = ("left", None)
        return
    try:
        total = allreduce_shares(share)
        out[rank] = ("ok", total.numpy().tolist())
    except Exception as exc:   # the others learn of the missing rank from the collective's time limit
        out[rank] = ("error", type(exc).__name__)
    dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_row_shares_allreduce_to_the_whole_profile(world):
    import oracle
    from paper_1306_2258_gb300 import workloads as wl
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_share_worker, args=(world, _free_port(), out, -1), nprocs=world, start_method="spawn",
                       join=True)
    mol = wl.random_walk_globule(240, 4, 77)
    ref = oracle.profile(mol.coords, mol.types, wl.form_factor_coefficients(4, 78), wl.q_grid(0.0, 0.8, 33))
    assert all(out[r][0] == "ok" for r in range(world))
    totals = [np.asarray(out[r][1]) for r in range(world)]
    for t in totals:
        assert np.array_equal(t, totals[0])            # the same bits on every rank
        assert np.max(np.abs(t - ref) / ref) <= 1e-11


def test_a_rank_that_leaves_makes_the_others_fail_not_hang():
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_share_worker, args=(2, _free_port(), out, 1), nprocs=2, start_method="spawn", join=True)
    assert out[1][0] == "left"
    assert out[0][0] == "error"


def _enc128(v):
    """A Python integer in [-2^127, 2^127) as int64 (low, high) halves of its two's complement."""
    v &= (1 << 128) - 1
    lo, hi = v & ((1 << 64) - 1), v >> 64
    return [lo - (1 << 64) if lo >= 1 << 63 else lo, hi - (1 << 64) if hi >= 1 << 63 else hi]


def _dec128(p):
    return (int(p[1]) << 64) + (int(p[0]) & ((1 << 64) - 1))


def _rank_values(rank, n=12):
    import random
    r = random.Random(900 + rank)
    return [r.randint(-(1 << 110), 1 << 110) for _ in range(n)]


def test_add_exact_is_integer_addition():
    from paper_1306_2258_gb300.shard import add_exact
    import random
    r = random.Random(5)
    for _ in range(50):
        k = r.randint(1, 9)
        vals = [[r.choice([r.randint(-(1 << 120), 1 << 120), r.randint(-3, 3), -(1 << 64), (1 << 64) - 1])
                 for _ in range(6)] for _ in range(k)]
        tot = add_exact([np.array([_enc128(v) for v in row], dtype=np.int64) for row in vals]).numpy()
        assert [_dec128(tot[j]) for j in range(6)] == [sum(row[j] for row in vals) for j in range(6)]


def _exact_worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    import torch
    import torch.distributed as dist

    from paper_1306_2258_gb300.shard import allreduce_exact
    dist.init_process_group("gloo", rank=rank, world_size=world)
    U = torch.as_tensor(np.array([_enc128(v) for v in _rank_values(rank)], dtype=np.int64))
    out[rank] = allreduce_exact(U).numpy().tolist()
    dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_exact_sums_allreduce_over_gloo_ranks(world):
    """Every rank's 128-bit sums (as a shard's sas_exact_sums) all-reduced as 32-bit limbs: every
    rank holds the exact integer total."""
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_exact_worker, args=(world, _free_port(), out), nprocs=world, start_method="spawn",
                       join=True)
    want = [sum(_rank_values(r)[j] for r in range(world)) for j in range(12)]
    for r in range(world):
        assert [_dec128(p) for p in out[r]] == want
