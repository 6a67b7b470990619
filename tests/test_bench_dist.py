"""The multi-rank arithmetic of bench.py on the CPU: two gloo ranks, each
with its own step time, agree on the max-over-ranks time, and the whole-job
value counts the bytes of every rank (weak scaling)."""
import os
import socket

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, times, out):
    import sys

    import torch.distributed as dist

    sys.path.insert(0, ROOT)
    import bench

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        t = bench.max_over_ranks(times[rank], dist, device="cpu")
        out.put((rank, t, bench.whole_job_gbs(world, 8 * 10**9, 4, t)))
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_world2():
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp

    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    times = [1.25, 2.0]
    procs = [ctx.Process(target=_rank, args=(r, 2, port, times, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [r[1] for r in res] == [2.0, 2.0]
    # 2 ranks x 8 GB x 4 steps in 2.0 s
    assert all(abs(r[2] - 32.0) < 1e-9 for r in res)


def test_single_rank_is_identity():
    import sys

    sys.path.insert(0, ROOT)
    import bench

    assert bench.max_over_ranks(3.5) == 3.5
    assert bench.whole_job_gbs(1, 10**9, 10, 2.0) == 5.0
