"""Multi-rank path of bench.py on CPU (gloo, world size 2).

The path does not shard: ranks run independent replicas and the reported time
is the maximum over ranks.  The reference arm runs on rank 0 only.
"""
import os
import socket

import pytest

torch = pytest.importorskip("torch")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import torch.distributed as dist
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        v = bench.aggregate_max(10.0 + 5.0 * rank, dist, "cpu")
        dist.barrier()
        q.put((rank, v))
    finally:
        dist.destroy_process_group()


def test_replicas_report_the_slowest_rank():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = dict(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert out == {0: 15.0, 1: 15.0}


def test_single_rank_needs_no_process_group():
    import bench
    assert bench.aggregate_max(3.5, None, "cpu") == 3.5


def test_reference_arm_prints_nothing_on_other_ranks(capsys):
    import argparse
    import bench
    bench.run_reference(argparse.Namespace(gpus=2, steps=1, warmup=3), rank=1)
    assert capsys.readouterr().out == ""
