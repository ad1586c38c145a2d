"""The multi-rank host logic of bench.py on CPU with the gloo backend (world size 2): every
rank gets its own problem instance, the timed region is the slowest rank's, and the job
throughput counts all ranks' queries.  No GPU and no data-path collective are involved."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import bench


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world, init_method=f"tcp://127.0.0.1:{port}")
    local_ms = 10.0 + 5.0 * rank           # rank 1 is the slower one
    total = bench.max_over_ranks(local_ms, dist, torch.device("cpu"))
    seed = bench.instance_seed(rank)
    out.put((rank, total, seed))
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_gloo():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    res.sort()
    assert [r[1] for r in res] == [15.0, 15.0]          # both see the slowest rank's time
    assert res[0][2] != res[1][2]                        # independent instances
    assert bench.job_throughput(1_000_000, world, 15.0 / 1) == pytest.approx(2 * 1e6 / 0.015)


def test_single_rank_is_local_time():
    assert bench.max_over_ranks(12.5, None) == 12.5
    assert bench.instance_seed(0) == 4                   # rank 0 answers the canonical mixed-1e8 seed
    assert bench.instance_seed(0, "mixed-1e7") == 2
