"""The multi-GPU replica path's host logic on CPU with two gloo ranks:
disjoint pairs per rank, max-over-ranks timing, whole-job throughput."""

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


def _worker(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        from paper_1501_02565_gb300.replicas import (max_over_ranks, rank_pair_indices,
                                                      whole_job_rate)
        idx = rank_pair_indices(rank, world, 5)
        t = 1.0 + rank            # rank 1 is the slower one
        tmax = max_over_ranks(t)
        rate = whole_job_rate(100.0, world, tmax)
        dist.barrier()
        q.put((rank, idx, tmax, rate))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks():
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    if root not in sys.path:
        sys.path.insert(0, root)
    ctx = mp.get_context("spawn")
    q = ctx.SimpleQueue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    res = sorted(q.get() for _ in range(2))
    (r0, i0, t0, v0), (r1, i1, t1, v1) = res
    assert set(i0).isdisjoint(i1) and len(i0) == len(i1) == 5
    assert t0 == t1 == 2.0                 # both ranks see the slowest time
    assert v0 == v1 == 100.0 * 2 / 2.0     # all ranks' units / max time


def test_single_process_identity():
    from paper_1501_02565_gb300.replicas import max_over_ranks, rank_pair_indices
    assert max_over_ranks(3.5) == 3.5
    assert rank_pair_indices(0, 1, 3) == [0, 1, 2]
    with pytest.raises(ValueError):
        rank_pair_indices(2, 2, 3)
