"""Sharding the batch of independent systems over ranks: the assignment
(complete, disjoint, balanced by the n^1.5 work model, deterministic), and the
end-of-batch exchange on two gloo ranks, where each rank factors its share
(with the oracle, on the CPU) and every rank must end up with the log dets of
all systems, equal to a single-process run."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

import gridgen  # noqa: E402
from paper_2409_14009_gb300.shard import partition_systems, work_estimate  # noqa: E402


@pytest.mark.parametrize("world", [1, 2, 3, 8])
def test_partition_is_complete_disjoint_and_balanced(world):
    probs = gridgen.batch_2d(count=200, kmin=16, kmax=96, seed=4)
    sizes = np.array([p.n for p in probs])
    parts = partition_systems(sizes, world)
    assert len(parts) == world
    allidx = np.concatenate(parts)
    assert np.array_equal(np.sort(allidx), np.arange(len(sizes)))
    w = work_estimate(sizes)
    loads = np.array([w[p].sum() for p in parts])
    # greedy LPT: no rank exceeds the mean by more than the largest system
    assert loads.max() <= loads.mean() + w.max() + 1e-9
    for p in parts:
        assert np.all(np.diff(p) > 0)
    assert all(np.array_equal(a, b) for a, b in zip(parts, partition_systems(sizes, world)))


def test_partition_of_equal_sizes_round_robins():
    parts = partition_systems([100] * 7, 3)
    assert [p.tolist() for p in parts] == [[0, 3, 6], [1, 4], [2, 5]]


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _batch():
    return gridgen.batch_2d(count=14, kmin=3, kmax=11, seed=17)


def _rank_main(rank, world, port, q):
    import sys
    sys.path.insert(0, ROOT)
    import oracle
    from paper_2409_14009_gb300.shard import gather_results, partition_systems
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        probs = _batch()
        mine = partition_systems([p.n for p in probs], world)[rank]
        lds, sts = [], []
        for i in mine:
            ref = oracle.reference(probs[i])
            lds.append(ref["fac"].logdet())
            sts.append(ref["fac"].info)
        ld, st = gather_results(dist, world, len(probs), mine, lds, sts)
        q.put((rank, mine.tolist(), ld.tolist(), st.tolist()))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_share_the_batch_and_gather_every_logdet():
    import oracle
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=180)
        assert p.exitcode == 0
    got = sorted(q.get(timeout=10) for _ in range(2))
    probs = _batch()
    single = [oracle.reference(p)["fac"].logdet() for p in probs]
    mine0, mine1 = got[0][1], got[1][1]
    assert sorted(mine0 + mine1) == list(range(len(probs))) and not set(mine0) & set(mine1)
    for rank, mine, ld, st in got:
        assert ld == single            # the same oracle arithmetic per system: bit for bit
        assert st == [0] * len(probs)
