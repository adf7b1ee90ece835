"""The multi-rank path of bench.py on CPU: two gloo ranks, each with its own
replica time, agree on the slowest rank's time and the whole-job throughput."""
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
    import torch.distributed as dist
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms = [2.5, 4.0][rank]
    m = bench.rank_max(ms, dist)
    out.put((rank, m, bench.job_throughput(3017, m, world)))
    dist.destroy_process_group()


def test_two_gloo_ranks_agree_on_max_time():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [m for _, m, _ in res] == [4.0, 4.0]
    assert res[0][2] == pytest.approx(2 * 3017 / 4.0e-3)


def test_single_rank_needs_no_process_group():
    import bench
    assert bench.rank_max(1.25) == 1.25
