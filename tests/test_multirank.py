"""Multi-rank timing logic of bench.py on CPU: two gloo ranks (replicas), the
max-over-ranks reduction, and the whole-job throughput of independent
replicas."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    import sys
    sys.path.insert(0, ROOT)
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        dist.barrier()
        # rank r "measured" (10 + 5 r) ms per step and (20 - r) ms end to end
        ms, e2e = bench.max_over_ranks(dist, [10.0 + 5.0 * rank, 20.0 - rank], torch.device("cpu"))
        q.put((rank, ms, e2e, bench.replica_throughput(1e9, world, ms)))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_take_the_max_and_sum_replicas():
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
    for rank, ms, e2e, gflops in got:
        assert ms == 15.0 and e2e == 20.0
        # two replicas of 1 GFLOP each within the slowest rank's 15 ms
        assert gflops == pytest.approx(2.0 / 0.015)


def test_single_rank_passthrough():
    import sys
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(None, [3.0, 4.0], None) == [3.0, 4.0]
    assert bench.replica_throughput(2e9, 1, 1000.0) == pytest.approx(2.0)
