"""The N > 1 path of bench.py on the CPU: two `gloo` ranks (replicas, no data
exchanged).  Each rank serves a disjoint seed range of the same queue size,
and every rank ends with the largest step time of all ranks, as bench.py
reports it."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, queue, out):
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    first = bench.rank_first_seed(rank, queue)
    seeds = list(range(first, first + queue))
    local_ms = 100.0 + 37.5 * rank                  # each rank's own step time
    ms = bench.max_over_ranks(local_ms, dist, "cpu")
    gathered = [None] * world
    dist.all_gather_object(gathered, seeds)
    out.put((rank, ms, gathered))
    dist.destroy_process_group()


def test_two_gloo_replicas():
    world, queue = 2, 5
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, world, port, queue, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, ms, gathered in res:
        assert ms == 137.5                           # the max over ranks on every rank
        assert set(gathered[0]).isdisjoint(gathered[1])
        assert gathered[0] == [2, 3, 4, 5, 6] and gathered[1] == [7, 8, 9, 10, 11]
