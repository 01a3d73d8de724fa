"""The multi-rank host logic of bench.py on CPU: two gloo ranks (weak scaling,
replicas only): disjoint image shards, max-over-ranks timing, barrier."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ws, r, local = bench.dist_env()
        shard = bench.shard_indices(r, ws, 16)
        bench.barrier()
        t = bench.max_over_ranks(1.0 + r)  # rank r "took" 1 + r seconds
        out.put((r, ws, local, shard, t))
    finally:
        dist.destroy_process_group()


@pytest.mark.timeout(120)
def test_two_gloo_ranks_shard_and_time():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=90) for _ in range(world))
    for p in procs:
        p.join(timeout=30)
        assert p.exitcode == 0
    shards = [set(x[3]) for x in res]
    assert all(len(s) == 16 for s in shards)
    assert not (shards[0] & shards[1])          # each rank draws its own images
    assert shards[0] | shards[1] == set(range(32))
    assert all(x[1] == world for x in res)
    assert all(x[4] == 2.0 for x in res)        # the slowest rank's time, on every rank


def test_reference_arm_runs_on_rank_zero_only(monkeypatch):
    # under torchrun the oracle's CPU timing runs once, on rank 0; other ranks exit 0 without work
    import argparse

    import bench
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setattr(bench, "make_inputs", lambda *a, **k: pytest.fail("rank 1 drew inputs"))
    assert bench.run_reference(argparse.Namespace(steps=3, warmup=3)) == 0
