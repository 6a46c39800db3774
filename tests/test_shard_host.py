"""Host side of the event-sharded likelihood, on CPU: the partition of the
events into group-aligned shards, and the all-gather of the ranks' group
partials in rank order over gloo with world size 2 and 3 (the GPU arithmetic is
covered by tests/test_gpu_shard.py with the ranks emulated on one device)."""
import os
import socket
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
G = 16384


def _shard():
    pytest.importorskip("torch")
    from paper_1706_01420_gb300 import shard
    return shard


@pytest.mark.parametrize("n", [0, 1, G - 1, G, G + 1, 5 * G + 7, 1_000_000, 50_000_000])
@pytest.mark.parametrize("world", [1, 2, 3, 4, 8])
def test_shards_partition_the_events_at_group_boundaries(n, world):
    shard = _shard()
    b = [shard.shard_bounds(n, r, world) for r in range(world)]
    assert b[0][0] == 0 and b[-1][1] == n
    for (lo, hi), (lo2, _) in zip(b, b[1:]):
        assert hi == lo2
    for lo, hi in b:
        assert lo <= hi and lo % G == 0
    rows = shard.shard_rows(n, world)
    assert sum(rows) == (n + G - 1) // G
    assert max(rows) - min(rows) <= 1


def test_bad_shard_arguments():
    shard = _shard()
    for args in ((10, 2, 2), (10, -1, 2), (10, 0, 0), (-1, 0, 1)):
        with pytest.raises(ValueError):
            shard.shard_bounds(*args)


def _worker(rank, world, port, n, width, q):
    sys.path.insert(0, ROOT)
    import torch
    import torch.distributed as dist
    from paper_1706_01420_gb300 import shard
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        rows = shard.shard_rows(n, world)
        lo = sum(rows[:rank])
        # rank r's partials: row g of the global order holds g + a / 100 in column a
        local = torch.tensor([[g + a / 100.0 for a in range(width)] for g in range(lo, lo + rows[rank])],
                             dtype=torch.float64).reshape(rows[rank], width)
        got = shard.gather_groups(local, rows, rank)
        q.put((rank, got.numpy().tolist()))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world,n", [(2, 5 * G + 7), (3, 2 * G)])
def test_gather_in_rank_order_gloo(world, n):
    torch = pytest.importorskip("torch")
    shard = _shard()
    width = 15
    mp = torch.multiprocessing.get_context("spawn")
    with socket.socket() as sk:
        sk.bind(("127.0.0.1", 0))
        port = sk.getsockname()[1]
    q = mp.Queue()
    procs = [mp.Process(target=_worker, args=(r, world, port, n, width, q)) for r in range(world)]
    for p in procs:
        p.start()
    got = dict(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    total = sum(shard.shard_rows(n, world))
    want = [[g + a / 100.0 for a in range(width)] for g in range(total)]
    for r in range(world):
        assert got[r] == want
