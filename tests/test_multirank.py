"""The N > 1 path of bench.py on CPU: world size 2 over gloo.  Every rank computes its own
energies (no collective on the data path); the only exchange is the max over ranks of the
timed region, and the whole-job value divides all ranks' units by that maximum."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    ws, r, local = bench.dist_init()
    dist.init_process_group("gloo", rank=r, world_size=ws)
    try:
        t_local = 1.0 + rank          # rank 1 is the slowest
        t = bench.max_over_ranks(t_local, dist, "cpu")
        out.put((r, ws, local, t, bench.job_value(4, ws, t)))
    finally:
        dist.destroy_process_group()


def test_two_ranks_take_the_slowest_time():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [r[:3] for r in res] == [(0, 2, 0), (1, 2, 1)]
    for r in res:
        assert r[3] == 2.0                    # max over ranks
        assert r[4] == pytest.approx(4.0)     # 4 energies x 2 ranks / 2 s


def test_single_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(3.5, None, "cpu") == 3.5
    assert bench.job_value(2, 1, 0.5) == 4.0
