"""The N > 1 benchmark path on CPU: two gloo ranks, max-over-ranks timing and the
whole-job (weak-scaling) rate. Every rank runs its own replica of the workload;
the only collective is the timing reduction (no data-path collective)."""
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


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    r, w, _ = bench.dist_env()
    ms = 100.0 + 50.0 * r                      # rank 1 is slower
    slow = bench.max_over_ranks(ms, w, "cpu")
    rate = bench.whole_job_rate(1000.0, w, slow)
    q.put((r, w, slow, rate))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_timing_reduction():
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
    assert [o[:2] for o in out] == [(0, 2), (1, 2)]
    for _, _, slow, rate in out:
        assert slow == 150.0                      # the max over ranks
        assert rate == pytest.approx(2 * 1000.0 / 0.150)   # all ranks' units / slowest time
