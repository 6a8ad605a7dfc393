"""Multi-rank host logic on CPU (gloo, world size 2): size-balanced sharding of
independent domains and the max-over-ranks timing reduction."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import synth_inputs as S
from paper_2411_09364_gb300.replicas import max_over_ranks, shard_domains

SIZES = [nx * ny * nz for nx, ny, nz in S.BATCH_DOMAINS]


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    mine = shard_domains(SIZES, world)[rank]
    gathered = [None] * world
    dist.all_gather_object(gathered, mine)
    t = max_over_ranks(float(10 + rank))
    if rank == 0:
        q.put((gathered, t))
    dist.barrier()
    dist.destroy_process_group()


def test_sharding_and_max_over_ranks_gloo_world2():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    gathered, t = q.get(timeout=120)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    flat = sorted(i for part in gathered for i in part)
    assert flat == list(range(len(SIZES)))                 # every domain exactly once
    loads = [sum(SIZES[i] for i in part) for part in gathered]
    assert max(loads) <= 1.1 * min(loads)                  # balanced
    assert t == 11.0                                       # max over ranks


def test_shard_domains_single_rank_and_more_ranks_than_domains():
    assert shard_domains([5, 3, 9], 1) == [[0, 1, 2]]
    parts = shard_domains([5, 3], 4)
    assert sorted(i for p in parts for i in p) == [0, 1] and sum(1 for p in parts if not p) == 2
