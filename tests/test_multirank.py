"""The benchmark's multi-GPU path is replicas only (independent instances per
rank, no data-path collective): check its host logic with two gloo ranks on
the CPU -- disjoint seeds per rank and the max-over-ranks step time."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    import torch
    import torch.distributed as dist
    import bench
    from paper_1407_5140_gb300 import workloads as W
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ds = bench.rank_instances(W.config1(), rank)
    seeds = torch.tensor([d["seed"] for d in ds], dtype=torch.int64)
    gathered = [torch.zeros_like(seeds) for _ in range(world)]
    dist.all_gather(gathered, seeds)
    t = bench.max_over_ranks(1.0 + rank, world)
    dist.barrier()
    out[rank] = ([sorted(set(g.tolist())) for g in gathered], t)
    dist.destroy_process_group()


def test_two_rank_replicas_use_disjoint_seeds_and_max_time():
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    procs = [ctx.Process(target=_worker, args=(r, world, port, out)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=300)
        assert p.exitcode == 0
    for r in range(world):
        per_rank, t = out[r]
        assert len(per_rank) == world
        assert not set(per_rank[0]) & set(per_rank[1])   # no seed shared between ranks
        assert t == float(world)                          # slowest rank's time
