"""Multi-GPU request dispatch, host logic only (no GPU): least-loaded
assignment by committed device bytes over fake per-device servers, and the
split of a request stream over two gloo ranks."""

import collections
import os
import socket

import pytest

from paper_1501_02565_gb300.dispatch import Dispatcher, rank_share


class FakeServer:
    """Stands in for serve.Server: requests are (name, bytes) and stay
    committed until finish() releases them."""

    def __init__(self):
        self.pending = collections.deque()
        self.committed = 0
        self.got = []

    def load(self):
        return self.committed

    def submit(self, req, **kw):
        self.pending.append(req)
        self.committed += req[1]
        self.got.append(req[0])

    def finish(self, name):
        for r in list(self.pending):
            if r[0] == name:
                self.pending.remove(r)
                self.committed -= r[1]

    def stop(self):
        return 0

    def stats(self):
        return {"requests": len(self.got)}


def test_least_loaded_by_bytes():
    a, b, c = FakeServer(), FakeServer(), FakeServer()
    d = Dispatcher([a, b, c])
    # one big request, then small ones: the small ones avoid the busy server
    assert d.submit(("big", 100))[1] == 0
    assert d.submit(("s1", 10))[1] == 1
    assert d.submit(("s2", 10))[1] == 2
    assert d.submit(("s3", 10))[1] == 1      # ties on bytes: fewest waiting, then lowest index
    assert d.submit(("s4", 10))[1] == 2
    a.finish("big")                          # server 0 drains
    assert d.submit(("s5", 50))[1] == 0
    assert d.assigned == [2, 2, 2]
    assert d.stop() == [0, 0, 0]
    assert [s["assigned"] for s in d.stats()] == [2, 2, 2]


def test_balances_bytes_over_a_mixed_stream():
    servers = [FakeServer() for _ in range(4)]
    d = Dispatcher(servers)
    sizes = [12, 3, 3, 30, 7, 7, 7, 2, 19, 5, 5, 11] * 10
    for i, b in enumerate(sizes):
        d.submit((f"r{i}", b))
    loads = [s.load() for s in servers]
    assert sum(loads) == sum(sizes)
    assert max(loads) - min(loads) <= max(sizes)


def test_rank_share_partitions_the_stream():
    for world in (1, 2, 3, 8):
        parts = [rank_share(101, r, world) for r in range(world)]
        flat = sorted(i for p in parts for i in p)
        assert flat == list(range(101))
        assert max(map(len, parts)) - min(map(len, parts)) <= 1
    with pytest.raises(ValueError):
        rank_share(10, 2, 2)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import torch
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        mine = rank_share(37, rank, world)
        # each rank "serves" its share; the ranks agree on the totals
        t = torch.tensor([len(mine), sum(mine)], dtype=torch.int64)
        dist.all_reduce(t)
        q.put((rank, mine, t.tolist()))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_split_a_request_stream():
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    if root not in sys.path:
        sys.path.insert(0, root)
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
    (r0, m0, t0), (r1, m1, t1) = out
    assert set(m0).isdisjoint(m1) and sorted(m0 + m1) == list(range(37))
    assert t0 == t1 == [37, sum(range(37))]
