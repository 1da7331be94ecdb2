"""The N > 1 plumbing of bench.py on CPU: two gloo ranks (127.0.0.1), each timing its own
replica, combine into the max-over-ranks time and the sum of the work of all ranks, which is
what the JSON line's whole-job value divides."""
import multiprocessing as mp
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    r, w, local = bench.dist_env()
    tmax, tsum = bench.reduce_max_sum(w, 1.5 + r, 100.0 * (r + 1), device="cpu")
    q.put((r, w, local, tmax, tsum))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_combine_time_and_work():
    pytest.importorskip("torch")
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [o[:3] for o in out] == [(0, 2, 0), (1, 2, 1)]
    for o in out:
        assert o[3] == 2.5            # the slower rank's time
        assert o[4] == 300.0          # both ranks' iterations
