"""Host logic of bench.py's multi-rank (replica) mode, on CPU with gloo, world size 2."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import torch
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    t = bench.max_over_ranks(10.0 + 5.0 * rank, dist, torch.device("cpu"))
    seeds = bench.rank_seed(1001, rank)
    dist.barrier()
    dist.destroy_process_group()
    q.put((rank, t, seeds))


def test_max_over_ranks_and_seeds_gloo():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [o[1] for o in out] == [15.0, 15.0]          # every rank sees the slowest time
    assert out[0][2] != out[1][2]                        # independent scans per rank


def test_single_rank_passthrough():
    import bench
    assert bench.max_over_ranks(3.5, None, None) == 3.5
