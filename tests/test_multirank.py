"""The N > 1 host logic of bench.py on CPU: two gloo ranks (one process per
rank, as torchrun launches them) aggregate the job's time as the slowest
rank's and its throughput as every rank's units over that time.  The solve
itself does not shard (replicas only), so this is the whole multi-rank path."""
import os
import socket

import pytest


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank(rank, world, port, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms = [12.5, 20.0][rank]
    units = [100, 140][rank]
    out = (bench.max_over_ranks(dist, ms, "cpu"), bench.sum_over_ranks(dist, units, "cpu"),
           bench.job_rate(dist, units, ms, "cpu"))
    dist.barrier()
    dist.destroy_process_group()
    q.put((rank, out))


def test_two_gloo_ranks_aggregate_max_time_and_summed_units():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = dict(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for r in (0, 1):
        mx, tot, rate = res[r]
        assert mx == 20.0 and tot == 240.0
        assert rate == pytest.approx(240.0 / 0.020)


def test_single_rank_is_identity():
    import bench
    assert bench.max_over_ranks(None, 3.5, "cpu") == 3.5
    assert bench.job_rate(None, 10, 5.0, "cpu") == pytest.approx(2000.0)
