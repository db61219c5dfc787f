"""The replica path of bench.py on CPUs: two gloo ranks (no GPU) agree on the
slowest rank's time and report the whole-job throughput."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    import torch.distributed as dist

    from paper_2309_01906_gb300 import replicas
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        assert replicas.world() == (world, rank)
        replicas.barrier()
        secs = 0.5 + rank                       # rank 1 is slower
        value, slowest = replicas.job_throughput(1000.0, secs)
        q.put((rank, value, slowest))
    finally:
        dist.destroy_process_group()


def test_two_ranks_agree_on_the_slowest_time():
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    got = sorted(q.get(timeout=10) for _ in range(2))
    for rank, value, slowest in got:
        assert slowest == 1.5
        assert value == pytest.approx(2 * 1000.0 / 1.5)


def test_single_process_is_its_own_job():
    from paper_2309_01906_gb300 import replicas
    assert replicas.world() == (1, 0)
    assert replicas.job_throughput(10.0, 2.0) == (5.0, 2.0)
