"""The multi-rank path of bench.py on CPU: two gloo ranks (127.0.0.1
rendezvous) take the slowest rank's time, aggregate whole-job throughput over
replicas, and the reference leg prints only on rank 0."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank_main(rank, world, port, q):
    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port), "RANK": str(rank),
                       "WORLD_SIZE": str(world), "LOCAL_RANK": str(rank)})
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    bench.barrier(world)
    slowest = bench.max_over_ranks(1.0 + rank, world)     # ranks report 1 ms and 2 ms
    value = bench.job_value(2 ** 24, world, slowest)
    q.put((rank, slowest, value))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_aggregate():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    got = sorted(q.get(timeout=10) for _ in range(2))
    for rank, slowest, value in got:
        assert slowest == pytest.approx(2.0)
        assert value == pytest.approx(2 * 2 ** 24 / 2e-3)


def test_reference_leg_silent_on_other_ranks(capsys):
    sys.path.insert(0, ROOT)
    import bench
    os.environ["RANK"] = "1"
    try:
        class A:
            warmup, steps, gpus = 1, 1, 2
        bench.run_reference(A())
    finally:
        os.environ.pop("RANK", None)
    assert capsys.readouterr().out == ""
