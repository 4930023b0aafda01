"""Continuous-batching server: every request's flow is bit-identical alone
and in the mix, admission respects the HBM budget, requests that arrive while
a batch runs join later batches."""

import time

import numpy as np
import pytest

from paper_1501_02565_gb300 import synth
from paper_1501_02565_gb300.native import EpicInterp
from paper_1501_02565_gb300.serve import Request, Server
from helpers import random_small_case

pytestmark = pytest.mark.gpu


def _requests():
    reqs = []
    for i in range(6):
        p = synth.config_pair(1, i)
        reqs.append(Request(p.C, p.matches, p.K, p.a, rid=len(reqs)))
    for i in range(6):
        C, M = random_small_case(700 + i, H=60 + 7 * i, W=90 + 11 * i, N=40 + 5 * i,
                                 c_lo=0.01, c_hi=1.0)
        reqs.append(Request(C, M, 8 + i, 1.0, rid=len(reqs)))
    p = synth.config_pair(2, 0)
    reqs.append(Request(p.C, p.matches, p.K, p.a, rid=len(reqs)))
    return reqs


def _alone(reqs):
    import torch
    eng = EpicInterp(0)
    out = []
    for r in reqs:
        f = eng.run(torch.from_numpy(r.C).cuda(), torch.from_numpy(r.matches).cuda(), r.K, r.a)
        eng.sync()
        out.append(f.cpu().numpy())
    eng.close()
    return out


def test_each_result_is_identical_alone_and_in_the_mix():
    reqs = _requests()
    ref = _alone(reqs)
    srv = Server(0, max_batch=8).start()
    # staggered arrivals: later requests arrive while earlier batches run
    for i, r in enumerate(reqs):
        srv.submit(r)
        if i % 4 == 3:
            time.sleep(0.002)
    for r in reqs:
        r.wait(timeout=60)
    assert srv.stop() == 0
    st = srv.stats()
    print("\n[serving]", st)
    assert st["requests"] == len(reqs)
    assert max(srv.batch_sizes) > 1      # requests were batched together
    for r, f in zip(reqs, ref):
        assert np.array_equal(r.flow.numpy(), f), r.rid


def test_admission_stays_within_the_hbm_budget():
    reqs = _requests()[:8]
    budget = 2 * max(r.device_bytes() for r in reqs)
    srv = Server(0, max_batch=8, hbm_budget=budget).start()
    for r in reqs:
        srv.submit(r)
    for r in reqs:
        r.wait(timeout=60)
    assert srv.stop() == 0
    assert srv.max_in_use <= budget
    assert len(srv.completed) == len(reqs)
    assert srv.steps >= 3                 # only a few requests fit at a time


def test_bad_request_is_refused_at_submission():
    srv = Server(0, max_batch=2)
    C = np.ones((10, 10), np.float32)
    with pytest.raises(ValueError):
        srv.submit(Request(C, np.array([[12, 1, 0, 0]], np.float32), 4, 1.0))
    C[3, 3] = np.nan
    with pytest.raises(ValueError):
        srv.submit(Request(C, np.array([[1, 1, 0, 0]], np.float32), 4, 1.0))
    srv.stop()


def test_host_buffer_batch_matches_device_batch():
    # the host-buffer entry point (copies in, one batched run, copies out)
    # gives the same flows as the device-buffer batch
    import torch
    from paper_1501_02565_gb300.native import EpicInterp
    pairs = [synth.config_pair(1, i) for i in range(9)] + [synth.config_pair(2, 0)]
    eng = EpicInterp(0, max_pairs=len(pairs))
    dev = [(torch.from_numpy(p.C).cuda(), torch.from_numpy(p.matches).cuda(), p.K, p.a,
            torch.empty((p.H, p.W, 2), dtype=torch.float32, device="cuda")) for p in pairs]
    eng.run_batch(dev)
    eng.sync()
    host = [(torch.from_numpy(p.C).pin_memory(), torch.from_numpy(p.matches).pin_memory(), p.K,
             p.a, torch.empty((p.H, p.W, 2), dtype=torch.float32).pin_memory()) for p in pairs]
    for _ in range(2):
        eng.run_batch_host(host)
        for d, hh in zip(dev, host):
            assert torch.equal(d[4].cpu(), hh[4])
    eng.close()


def test_streamed_host_batches_match_device_batches():
    import torch
    # three different batches submitted back to back (two in flight at a
    # time, the third waits for the first's downloads), one sync at the end
    pairs = [synth.config_pair(1, i) for i in range(6)]
    batches = [pairs[0:2], pairs[2:5], pairs[5:6]]
    eng = EpicInterp(0, max_pairs=4)
    expect = []
    for b in batches:
        dev = [(torch.from_numpy(p.C).cuda(), torch.from_numpy(p.matches).cuda(), p.K, p.a,
                torch.empty((p.H, p.W, 2), dtype=torch.float32, device="cuda")) for p in b]
        eng.run_batch(dev)
        eng.sync()
        expect.append([d[4].cpu() for d in dev])
    for _ in range(2):
        host = [[(torch.from_numpy(p.C).pin_memory(), torch.from_numpy(p.matches).pin_memory(),
                  p.K, p.a, torch.full((p.H, p.W, 2), float("nan")).pin_memory()) for p in b]
                for b in batches]
        for h in host:
            eng.submit_batch_host(h)
        eng.sync()
        for h, ex in zip(host, expect):
            for hh, e in zip(h, ex):
                assert torch.equal(hh[4], e)
    eng.close()


def test_dispatcher_over_the_devices_matches_single_runs():
    # the dispatcher over every visible device (one on this machine): each
    # request lands on the least-loaded server and its flow is the one a
    # single run gives
    import torch
    from paper_1501_02565_gb300.dispatch import Dispatcher
    reqs = _requests()[:6]
    ref = _alone(reqs)
    d = Dispatcher.on_devices(range(torch.cuda.device_count()), max_batch=4)
    for r in reqs:
        d.submit(r)
    for r in reqs:
        r.wait(timeout=60)
    assert all(s == 0 for s in d.stop())
    assert sum(st["assigned"] for st in d.stats()) == len(reqs)
    for r, f in zip(reqs, ref):
        assert np.array_equal(r.flow.numpy(), f), r.rid
