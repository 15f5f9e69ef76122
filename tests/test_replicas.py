"""The benchmark's multi-process path on CPU: two gloo ranks.

Under torchrun every rank runs its own replica of the solve (the path has no
exchange step); the job's time is the slowest rank's, and the throughput
counts the work of all ranks.  This checks the rank reduction and the
environment parsing with world size 2, without a GPU.
"""
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


def _rank_main(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ws, r, local = bench._dist()
        out = bench.worst_over_ranks([10.0 + rank, 5.0 - rank])
        q.put((r, ws, local, out))
    finally:
        dist.destroy_process_group()


def test_worst_over_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [r[0] for r in res] == [0, 1]
    for r, ws, local, out in res:
        assert ws == 2 and local == r
        assert out == [11.0, 5.0]


def test_single_process_is_unchanged():
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    assert bench.worst_over_ranks([3.0, 4.0]) == [3.0, 4.0]
