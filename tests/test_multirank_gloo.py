"""The host side of the N > 1 bench path on two CPU ranks over gloo (no GPU): the timed region's
length is the slowest rank's (maximum over ranks), the job's rate counts the points of every rank
(weak scaling: each rank advances its own replica), and the reference arm runs on rank 0 alone
while the other ranks exit 0 without work."""
import argparse
import socket

import pytest

mp = pytest.importorskip("torch.multiprocessing")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    import torch.distributed as dist

    import bench
    dist.init_process_group("gloo", init_method="tcp://127.0.0.1:%d" % port, rank=rank, world_size=world)
    seconds = bench.max_over_ranks(1.5 + rank, dist, "cpu")       # rank 1 is the slow one
    rate = bench.job_rate(1000, 5, world, seconds)
    rc = None
    if rank != 0:
        args = argparse.Namespace(impl="reference", workload="tgv", n=256, scheme=2, steps=2, warmup=1,
                                  gpus=world, seed=0)
        rc = bench.run_reference(args, rank)
    dist.barrier()
    dist.destroy_process_group()
    q.put((rank, seconds, rate, rc))


def test_two_gloo_ranks_take_the_slowest_time_and_count_every_rank():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=180) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, seconds, rate, rc in out:
        assert seconds == 2.5                               # max(1.5, 2.5) on both ranks
        assert rate == pytest.approx(1000 * 3 * 5 * 2 / 2.5 / 1e6)
    assert out[1][3] == 0                                   # reference arm: rank 1 exits at once


def test_single_process_reduction_is_the_identity():
    import bench
    assert bench.max_over_ranks(3.25, None, "cpu") == 3.25
    assert bench.job_rate(16777216, 5, 1, 0.05) == pytest.approx(16777216 * 15 / 0.05 / 1e6)
