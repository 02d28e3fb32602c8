"""The multi-rank host logic of the benchmark on CPU: two gloo ranks (no GPU)."""
import os
import socket

import pytest


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, results):
    import torch.distributed as dist

    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        # each rank scans its own text (weak scaling): ranks differ in their seed only
        local_s = 2.0 if rank == 0 else 3.0
        total, value = bench.job_throughput(local_s, 1000, 10, world, "cpu")
        results[rank] = (total, value)
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_rank():
    mp = pytest.importorskip("torch.multiprocessing")
    ctx = mp.get_context("spawn")
    port = _free_port()
    with ctx.Manager() as mgr:
        results = mgr.dict()
        procs = [ctx.Process(target=_rank_main, args=(r, 2, port, results)) for r in range(2)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(120)
        assert all(p.exitcode == 0 for p in procs)
        got = dict(results)
    # the job takes as long as its slowest rank, and counts the bases of both ranks
    for r in (0, 1):
        total, value = got[r]
        assert total == pytest.approx(3.0)
        assert value == pytest.approx(2 * 1000 * 10 / 3.0 / 1e9)


def test_single_rank_needs_no_process_group():
    import bench
    total, value = bench.job_throughput(0.5, 256, 4, 1)
    assert total == 0.5 and value == pytest.approx(256 * 4 / 0.5 / 1e9)


def test_each_rank_scans_its_own_text():
    import bench
    a = bench.make_workload(0, 1 << 14, 50)
    b = bench.make_workload(1, 1 << 14, 50)
    assert a.text.size == b.text.size and not (a.text == b.text).all()
