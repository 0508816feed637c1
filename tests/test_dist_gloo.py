"""The multi-rank host logic (paper_1712_04718_gb300.sharding) on two CPU ranks (gloo): the
ensemble's systems are split over the ranks without overlap or gaps and with
balanced cost, every rank computing the same assignment, and the timing
reduction returns the slowest rank's time on every rank."""
import math
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_1712_04718_gb300 import sharding, systems


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _ensemble_sizes():
    # the 64-box ensemble's box edges, atom counts and grids, without coordinates
    rng = __import__("numpy").random.default_rng(999)
    Ls = rng.uniform(3.0, 7.0, size=64)
    Ms = [systems.smooth7(math.ceil(L / 0.12)) for L in Ls]
    Ns = [3 * round(33.4 * L ** 3) for L in Ls]
    return Ns, Ms


def _worker(rank, ws, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        Ns, Ms = _ensemble_sizes()
        costs = [sharding.system_cost(n, m, 8) for n, m in zip(Ns, Ms)]
        parts = sharding.partition_systems(costs, ws)
        gathered = [None] * ws
        dist.all_gather_object(gathered, parts[rank])
        slowest = sharding.max_over_ranks(10.0 * (rank + 1), ws, "cpu")
        out.put((rank, gathered, slowest, parts))
    finally:
        dist.destroy_process_group()


def test_partition_and_max_over_two_gloo_ranks():
    ws = 2
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, ws, port, out)) for r in range(ws)]
    for p in procs:
        p.start()
    res = [out.get(timeout=120) for _ in range(ws)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    res.sort()
    Ns, Ms = _ensemble_sizes()
    costs = [sharding.system_cost(n, m, 8) for n, m in zip(Ns, Ms)]
    for rank, gathered, slowest, parts in res:
        assert slowest == 20.0                      # the slowest rank's time on every rank
        assert gathered == res[0][3]                # every rank computed the same assignment
        assert gathered[rank] == parts[rank]
    parts = res[0][3]
    flat = sorted(i for p in parts for i in p)
    assert flat == list(range(64))                  # no overlap, no gap
    loads = [sum(costs[i] for i in p) for p in parts]
    assert max(loads) <= 1.05 * min(loads)          # balanced


def test_partition_single_rank_and_more_ranks_than_systems():
    assert sharding.partition_systems([3.0, 1.0, 2.0], 1) == [[0, 1, 2]]
    parts = sharding.partition_systems([3.0, 1.0], 4)
    assert sorted(i for p in parts for i in p) == [0, 1] and sum(1 for p in parts if not p) == 2
    assert sharding.max_over_ranks(1.5, 1, "cpu") == 1.5


def test_shard_covers_the_ensemble_once():
    Ns, Ms = _ensemble_sizes()
    ws = 3
    got = sorted(i for r in range(ws) for i in sharding.shard(Ns, Ms, 8, ws, r))
    assert got == list(range(64))
