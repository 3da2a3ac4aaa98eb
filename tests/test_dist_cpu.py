"""The multi-process path of bench.py on CPU (gloo, world size 2): one
process per rank, a barrier around the timed region, and the step time taken
as the maximum over ranks (each rank counts its own replica of the
workload, so there is no data-path collective)."""
import multiprocessing as mp
import os
import socket

import pytest


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, ws, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws),
                      LOCAL_RANK=str(rank))
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import torch.distributed as dist

    import bench
    ws_, rank_, _ = bench.dist_setup("gloo")
    bench.barrier(ws_)
    step = bench.allreduce_max(0.5 + rank_, ws_)  # the slower rank sets the step time
    bench.barrier(ws_)
    q.put((rank_, ws_, step))
    dist.destroy_process_group()


def test_two_ranks_take_the_max_step_time():
    pytest.importorskip("torch")
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    out = sorted(q.get(timeout=10) for _ in range(2))
    assert out == [(0, 2, 1.5), (1, 2, 1.5)]


def test_single_process_needs_no_process_group():
    import bench
    assert bench.allreduce_max(3.0, 1) == 3.0
    bench.barrier(1)
