"""Sharded counting (ttc_count_shard): every static triangle is counted on
its own (Alg. 1), so each bin of the triangle list can be cut into slices
that different GPUs or processes count.  Checked on the GPU: the shards'
counts sum to the whole graph's, for several shard counts and graphs whose
triangles fill every bin (light, one warp, one CTA, flat); and two processes
on one GPU, each counting its shard of the same graph, reach the oracle's
counts through the gloo sum of paper_2106_02762_gb300.shard."""
import multiprocessing as mp
import os
import socket

import numpy as np
import pytest

import oracle
from paper_2106_02762_gb300 import synth, ttc

pytestmark = pytest.mark.gpu

BIG = 1 << 40
DELTAS = [(3600, 1800, 1800), (BIG, BIG, BIG), (200000, 150000, 120000)]


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()


def _with_huge(big):
    """A triangle {0, 1, 2} with big, 1500 and 1500 edges on its pairs (its
    two enumerated lists exceed one CTA: the flat path) plus a small
    power-law graph on other ids."""
    rng = np.random.default_rng(11)
    src, dst = [], []
    for (a, b), k in zip(((0, 1), (0, 2), (1, 2)), (big, 1500, 1500)):
        flip = rng.integers(0, 2, size=k).astype(bool)
        src.append(np.where(flip, b, a))
        dst.append(np.where(flip, a, b))
    s, d, t = synth.large_plain(scale=0.002)
    src = np.concatenate(src + [s.astype(np.int64) + 3]).astype(np.uint32)
    dst = np.concatenate(dst + [d.astype(np.int64) + 3]).astype(np.uint32)
    tt = np.concatenate([rng.integers(0, 1 << 22, size=big + 3000), t]).astype(np.int64)
    return src, dst, tt


@pytest.mark.parametrize("which", ["power_law", "huge_narrow", "huge_wide"])
def test_shards_sum_to_the_whole(which):
    if which == "power_law":
        s, d, t = synth.large_plain(scale=0.003)
    else:
        s, d, t = _with_huge(1500 if which == "huge_narrow" else 70000)
    g = ttc.Graph(s, d, t)
    info = g.info()
    assert info["tau_light"] and info["tau_hwarp"] and info["tau_hcta"]
    if which != "power_law":
        assert info["tau_huge"] >= 1
    whole = g.count_batch(DELTAS)
    assert (whole == oracle.count(s, d, t, DELTAS)).all()
    for n in (1, 2, 3, 5):
        parts = [g.count_shard(DELTAS, r, n) for r in range(n)]
        assert (sum(p.astype(object) for p in parts) == whole.astype(object)).all(), n
    # a shard of a single query equals the same shard of the batch
    assert (g.count_shard(DELTAS[1:2], 1, 3)[0] == g.count_shard(DELTAS, 1, 3)[1]).all()
    g.free()


def test_shard_arguments_checked():
    s, d, t = synth.tiny_plain()
    g = ttc.Graph(s, d, t)
    for shard, n in ((0, 0), (2, 2), (5, 3)):
        with pytest.raises(ttc.TTCError, match="INVALID"):
            g.count_shard(DELTAS, shard, n)
    g.free()
    gs = ttc.Graph(s, d, t, streamed=True)
    with pytest.raises(ttc.TTCError, match="INVALID"):
        gs.count_shard(DELTAS, 0, 2)
    gs.free()


def _free_port():
    so = socket.socket()
    so.bind(("127.0.0.1", 0))
    port = so.getsockname()[1]
    so.close()
    return port


def _rank(rank, ws, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws))
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import torch
    import torch.distributed as dist

    from paper_2106_02762_gb300 import shard, synth, ttc
    torch.cuda.set_device(0)
    dist.init_process_group("gloo")
    s, d, t = _with_huge(1500)
    g = ttc.Graph(s, d, t)
    mine = g.count_shard(DELTAS, rank, ws)
    total = shard.count_sharded(g, DELTAS, rank, ws)
    g.free()
    q.put((rank, mine.tolist(), total.tolist()))
    dist.barrier()
    dist.destroy_process_group()


def test_two_processes_count_their_shards():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(300)
        assert p.exitcode == 0
    out = dict((r, (np.array(m, dtype=np.uint64), np.array(tot, dtype=np.uint64)))
               for r, m, tot in (q.get(timeout=10) for _ in range(2)))
    s, d, t = _with_huge(1500)
    want = oracle.count(s, d, t, DELTAS)
    assert (out[0][1] == want).all() and (out[1][1] == want).all()
    assert ((out[0][0].astype(object) + out[1][0].astype(object)) == want.astype(object)).all()
    assert out[0][0].sum() > 0 and out[1][0].sum() > 0
