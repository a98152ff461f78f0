"""The N > 1 path of bench.py on CPU: replicas joined by a gloo process group.

Every rank solves its own copy of the sequence (no data-path collective); the
only exchange is the max over ranks of the timed region, after which the
whole-job figure is that time over all systems of all ranks.  Two ranks here,
with unequal elapsed times, must agree on the maximum and on the whole-job
ms per system."""

import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist          # noqa: E402
import torch.multiprocessing as mp        # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        r, w, lr = bench.dist_env()
        steps = 5
        elapsed = 100.0 + 50.0 * rank        # rank 1 is the slow one
        T, value = bench.aggregate(elapsed, steps, w, dist)
        q.put((r, w, lr, T, value))
    finally:
        dist.destroy_process_group()


def test_two_replicas_take_the_max_and_count_all_systems():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [o[0] for o in out] == [0, 1] and all(o[1] == 2 and o[2] == o[0] for o in out)
    for _, _, _, T, value in out:
        assert T == 150.0
        assert value == pytest.approx(150.0 / (5 * 2))


def test_single_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    T, value = bench.aggregate(80.0, 4, 1, None)
    assert T == 80.0 and value == 20.0
