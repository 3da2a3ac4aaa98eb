"""The multi-process path on CPU (gloo, world size 2): bench.py's barrier
around the timed region and step time taken as the maximum over ranks, and
the one exchange of a sharded count, the exact sum of the ranks' uint64
counts (paper_2106_02762_gb300.shard)."""
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


def _sum_rank(rank, ws, port, q, rows):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws),
                      LOCAL_RANK=str(rank))
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import numpy as np
    import torch.distributed as dist

    from paper_2106_02762_gb300 import shard
    dist.init_process_group("gloo")
    res = []
    for row in rows:
        mine = np.array(row[rank], dtype=np.uint64)
        try:
            res.append(shard.allreduce_counts(mine).tolist())
        except OverflowError:
            res.append("overflow")
    q.put((rank, res))
    dist.destroy_process_group()


def test_two_ranks_sum_uint64_counts_exactly():
    pytest.importorskip("torch")
    top = (1 << 64) - 1
    rows = [
        # counts that need all 64 bits, and carries out of the low halves
        [[top - 5, 0xFFFFFFFF, 7, 0, 1 << 63, 3, 0xFFFFFFFF, 1], [5, 1, 0, 0, (1 << 63) - 1, 4, 0xFFFFFFFF, 2]],
        # a total of 2^64 is an overflow, not a wrap to zero
        [[top, 0, 0, 0, 0, 0, 0, 0], [1, 0, 0, 0, 0, 0, 0, 0]],
    ]
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_sum_rank, args=(r, 2, port, q, rows)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    out = dict(q.get(timeout=10) for _ in range(2))
    want0 = [a + b for a, b in zip(rows[0][0], rows[0][1])]
    assert max(want0) < 1 << 64
    for r in (0, 1):
        assert out[r][0] == want0
        assert out[r][1] == "overflow"
