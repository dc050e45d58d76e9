"""The N>1 path of bench.py on CPU ranks (gloo): each rank processes its own
pairs (replicas, no data-path collective); the job's time is the slowest
rank's and its rate counts every rank's pairs."""
import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, ws, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws))
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    ms = [120.0, 95.0][rank]          # rank 0 is the slowest
    m = bench.max_over_ranks(ms, dist, "cpu")
    rate = bench.job_throughput(10, ws, m)
    q.put((rank, m, rate))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time_and_count_all_pairs():
    ws, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, ws, port, q)) for r in range(ws)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    out = sorted(q.get(timeout=10) for _ in range(ws))
    for rank, m, rate in out:
        assert m == 120.0
        assert rate == pytest.approx(20 / 0.120)


def test_single_rank_needs_no_collective():
    import bench
    assert bench.max_over_ranks(3.5, None, "cpu") == 3.5
    assert bench.job_throughput(4, 1, 500.0) == pytest.approx(8.0)
