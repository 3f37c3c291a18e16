"""The replica path of the benchmark on two gloo ranks (CPU): every rank
sees the slowest rank's times, and the whole-job rate counts every rank's
work over that time."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as sk:
        sk.bind(("127.0.0.1", 0))
        return sk.getsockname()[1]


def _rank_main(rank, world, port, q):
    import torch.distributed as tdist
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    tdist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms, e2e = bench.replica_max([100.0 + 50.0 * rank, 300.0 - 100.0 * rank], "cpu")
        q.put((rank, ms, e2e, bench.whole_job_rate(1000, world, ms)))
    finally:
        tdist.destroy_process_group()


def test_two_replicas_take_the_slowest_time():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    got = sorted(q.get(timeout=10) for _ in range(2))
    for rank, ms, e2e, rate in got:
        assert ms == 150.0 and e2e == 300.0
        assert rate == pytest.approx(2 * 1000 / 0.150)
