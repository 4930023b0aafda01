"""Throughput and latency benchmark of the GB300 sparse-to-dense interpolator.

One step = the whole interpolator (relaxation, match graph, K-NN + LA fit,
write-out) over one batch of synthetic pairs, launched as one batched run
through the C ABI and replayed from a captured CUDA graph.  The headline
workload is the mixed-size batch: 64 pairs with sizes drawn from
{640x480, 1024x436, 1242x375, 1920x1080}, N = P/100 clipped to [2000, 20000],
K in {64, 100, 128}, 10-80 regions, a = 1 (~53 Mpix and ~0.7 GB of inputs
and outputs per step, far above the 129 MB L2, so consecutive steps do not
run from cache).

Prints one JSON line (rank 0).  Keys beyond the common ones:
  roofline      the dominant kernel's achieved rate vs the measured HBM peak;
                kernel times from CUDA events the library records between
                its kernels over a second timed region of the same steps
                (plain launches: stage events are not recorded inside a
                replayed graph); traffic from the committed ncu summary (null
                if the kernel source changed since the capture)
  stages        the same figures for every kernel
  e2e           same metric through the host-buffer API: every step uploads
                its inputs from pinned host memory and downloads its flows
                inside the timed region (epic_interp_submit_batch_host per
                step, one epic_interp_sync); blocking_value waits per step
  plain         the one-pair-at-a-time GPU path on the headline pairs
                (plain launches, and replayed graphs)
  configs       per configuration: the single pair (256x128), Sintel-shaped
                (1024x436) and KITTI-shaped (1242x375) pairs, each as
                one-pair latency p50/p99 and as a batch of 32 distinct pairs
  served        the serving stream: 2000 Poisson requests (sizes uniform over
                {640x480, 1024x436, 1242x375, 2048x1024}, N up to 30000,
                K = 100), at several arrival rates from under- to over-load,
                through the continuous-batching server and through the same
                server limited to one request per step; p50/p99 latency and
                Mpix/s at every rate
  pruned        the headline batch with the NW consistency pruning of
                Sec. 4.1 (two passes per run)
  exact         the exact per-pixel variant of Sec. 5.2 (geodesic and
                Euclidean) on one Sintel-shaped pair
  gradient_cost the image-gradient cost map (Table 2) of 32 frames vs HBM
  refine        the variational refinement (Sec. 4) of one Sintel-shaped pair
  cpu_baseline  the FP64 CPU oracle on the host cores, on a bounded sample
  clocks        nvidia-smi samples taken during the timed region

--impl reference runs the oracle itself as the reference arm.
Multi-GPU (torchrun): independent replicas, one batch of distinct pairs per
rank, no collective on the data path ("scaling": "weak").
"""

from __future__ import annotations

import argparse
import concurrent.futures as cf
import glob
import hashlib
import json
import multiprocessing as mp
import os
import re
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "interpolated Mpix/s and p50/p99 latency, served+batched vs plain GPU, at 1e-3 px"
WORKLOAD = ("mixed-size batch: 64 pairs, sizes from {640x480, 1024x436, 1242x375, 1920x1080}, "
            "N = P/100 in [2000, 20000], K in {64, 100, 128}, 10-80 regions, a = 1")
HEADLINE_CONFIG = 4
PAPER_MPIX_S = 1024 * 436 / 0.25 / 1e6   # Sec. 5.4: 0.25 s per 1024x436 pair, 1 core
STAGES = ("prepare", "relax", "edges", "scatter", "knn_fit", "writeout")
KERNEL_SRC = {
    "prepare": "k_prepare.cu", "relax": "k_relax.cu", "edges": "k_graph.cu",
    "scatter": "k_graph.cu", "knn_fit": "k_knn_fit.cu", "writeout": "k_writeout.cu",
}


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--batch", type=int, default=64, help="pairs per headline step")
    ap.add_argument("--impl", default="ours", choices=("ours", "reference"))
    ap.add_argument("--cpu-threads", type=int, default=0)
    ap.add_argument("--requests", type=int, default=2000, help="requests per serving rate")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-tune", action="store_true", help="skip the tile autotuner")
    ap.add_argument("--no-exact", action="store_true", help="skip the exact-variant leg")
    ap.add_argument("--no-serve", action="store_true", help="skip the serving sweep")
    ap.add_argument("--no-extra", action="store_true",
                    help="headline, stages and e2e only (for profiling runs)")
    return ap.parse_args()


# ---------------------------------------------------------------------------
# inputs (generated on the host in parallel; spawned workers, started before
# any GPU work)
# ---------------------------------------------------------------------------

def _gen(args):
    from paper_1501_02565_gb300 import synth
    config, index = args
    return synth.config_pair(config, index)


def gen_pairs(jobs, workers):
    """config_pair(c, i) for every (c, i) of `jobs`, in order."""
    if workers <= 1 or len(jobs) <= 2:
        return [_gen(j) for j in jobs]
    ctx = mp.get_context("spawn")
    with cf.ProcessPoolExecutor(max_workers=workers, mp_context=ctx) as ex:
        return list(ex.map(_gen, jobs, chunksize=1))


def rank_jobs(config, n, rank, world):
    from paper_1501_02565_gb300.replicas import rank_pair_indices
    return [(config, i) for i in rank_pair_indices(rank, max(world, rank + 1), n)]


# ---------------------------------------------------------------------------
# workload accounting (algorithmic bytes per unit; see the design notes)
# ---------------------------------------------------------------------------

def algorithmic_bytes(stage, pairs, n_edges):
    P = sum(p.P for p in pairs)
    N = sum(p.N for p in pairs)
    if stage == "relax":        # read C, write (D, L)
        return 12.0 * P
    if stage == "edges":        # read (D, L) and C
        return 12.0 * P
    if stage == "writeout":     # read L, write flow (u, v)
        return 12.0 * P
    if stage == "prepare":      # read matches, write seed bins
        return 20.0 * N
    if stage == "scatter":      # read edge table, write both adjacency entries
        return 28.0 * n_edges
    if stage == "knn_fit":      # per match: K neighbour records (16 B) and
        # their adjacency rows (deg x 8 B), plus the 32 B model
        deg = 2.0 * n_edges / max(N, 1)
        return sum(p.N * (min(p.K, p.N) * (16.0 + deg * 8.0) + 32.0) for p in pairs)
    raise KeyError(stage)


def kernel_sha(stage):
    path = os.path.join(ROOT, "paper_1501_02565_gb300", "csrc", KERNEL_SRC[stage])
    h = hashlib.sha256(open(path, "rb").read()).hexdigest()
    return h[:16]


def committed_traffic(stage, workload):
    """dram bytes per launch from a committed ncu summary of this kernel on
    this workload, if its source hash still matches."""
    for f in glob.glob(os.path.join(ROOT, "profiles", "*.md")):
        txt = open(f).read()
        m = re.search(r"traffic_bytes_per_launch\[%s,%s\]:\s*([0-9.eE+]+)\s+src=([0-9a-f]+)"
                      % (stage, re.escape(workload)), txt)
        if m and m.group(2) == kernel_sha(stage):
            return float(m.group(1)), os.path.relpath(f, ROOT)
    return None, None


def measured_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        # raw samples: $EPIC_CLOCKS_DIR if set (to keep them), else the temp dir
        out_dir = os.environ.get("EPIC_CLOCKS_DIR") or tempfile.gettempdir()
        self.path = os.path.join(out_dir, f"epic_clocks_rank{gpu_index}.csv")

    def start(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "50"],
                stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.fh.close()
        rows = []
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                rows.append((float(parts[1]), float(parts[2]), parts[5:9]))
            except ValueError:
                continue
        if not rows:
            return None
        sm = [r[0] for r in rows]
        reasons = set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for r in rows:
            for nm, v in zip(names, r[2]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": max(r[1] for r in rows),
                "reasons": sorted(reasons), "samples": len(rows)}


# ---------------------------------------------------------------------------
# CPU oracle (baseline leg and reference arm)
# ---------------------------------------------------------------------------

def oracle_pass(pairs, threads):
    import oracle
    oracle.build()
    t0 = time.perf_counter()
    with cf.ThreadPoolExecutor(max_workers=threads) as ex:
        list(ex.map(lambda p: oracle.interp(p.C, p.matches, p.K, p.a)["flow"].shape, pairs))
    return time.perf_counter() - t0


def cpu_threads(args):
    if args.cpu_threads > 0:
        return args.cpu_threads
    return max(1, min(os.cpu_count() or 1, 16))


def reference_sample(pairs, threads):
    """A bounded sample of the headline batch for the oracle: its first
    pairs (mixed sizes, as drawn), one per thread, so that a step takes a few
    seconds of wall time on the host cores."""
    return list(pairs[: min(len(pairs), threads)])


def run_reference(args, rank, world):
    if rank != 0:
        return 0
    threads = cpu_threads(args)
    pairs = gen_pairs(rank_jobs(HEADLINE_CONFIG, args.batch, 0, 1), threads)
    sample = reference_sample(pairs, threads)
    for _ in range(args.warmup):
        oracle_pass(sample, threads)
    t = 0.0
    for _ in range(args.steps):
        t += oracle_pass(sample, threads)
    px = sum(p.P for p in sample) * args.steps
    value = px / t / 1e6
    desc = (f"{len(sample)} pairs of the headline batch per step ({sum(p.P for p in sample)} "
            f"pixels), one pair per thread")
    line = {
        "impl": "reference", "metric": METRIC, "value": value,
        "unit": "Mpix/s", "n_gpus": args.gpus, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * t / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "pairs_per_step": len(sample)},
        "cpu_baseline": {"kind": "oracle", "cores": min(threads, len(sample)), "value": value,
                         "unit": "Mpix/s", "sample": desc},
        "e2e": {"value": value, "unit": "Mpix/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------------------
# GPU helpers
# ---------------------------------------------------------------------------

def device_items(pairs, dev):
    import torch
    return [(torch.from_numpy(p.C).to(dev), torch.from_numpy(p.matches).to(dev), p.K, p.a,
             torch.empty((p.H, p.W, 2), dtype=torch.float32, device=dev)) for p in pairs]


def engine_for(pairs, device, **cfg):
    from paper_1501_02565_gb300.native import EpicInterp
    return EpicInterp(device, max_pairs=len(pairs), max_H=max(p.H for p in pairs),
                      max_W=max(p.W for p in pairs), max_N=max(p.N for p in pairs),
                      max_K=max(p.K for p in pairs), **cfg)


def time_batched(eng, items, steps, warmup, stream):
    """ms per step of `steps` batched runs on `stream` (CUDA events)."""
    import torch
    with torch.cuda.stream(stream):
        for _ in range(max(warmup, 3)):
            eng.run_batch(items, stream=stream)
        stream.synchronize()
        eng.sync()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            eng.run_batch(items, stream=stream)
        e1.record(stream)
        stream.synchronize()
    eng.sync()
    return e0.elapsed_time(e1) / steps


def time_plain(eng, items, stream):
    """One pair per run, back to back: per-pair latency (ms, CUDA events)
    and the throughput of the whole sequence (Mpix/s)."""
    import torch
    with torch.cuda.stream(stream):
        for it in items[:4]:
            eng.run_batch([it], stream=stream)
        stream.synchronize()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in items]
        t0 = torch.cuda.Event(enable_timing=True)
        t1 = torch.cuda.Event(enable_timing=True)
        t0.record(stream)
        for it, (a0, a1) in zip(items, ev):
            a0.record(stream)
            eng.run_batch([it], stream=stream)
            a1.record(stream)
        t1.record(stream)
        stream.synchronize()
    eng.sync()
    lat = [a0.elapsed_time(a1) for a0, a1 in ev]
    px = sum(it[0].numel() for it in items)
    return lat, px / (t0.elapsed_time(t1) / 1e3) / 1e6


def plain_line(lat, value):
    return {"value": value, "unit": "Mpix/s", "latency_ms_p50": float(np.percentile(lat, 50)),
            "latency_ms_p99": float(np.percentile(lat, 99)), "pairs": len(lat)}


def config_line(pairs, device, rules, steps, warmup, stream):
    """One configuration: batched (graph replay) throughput over its pairs and
    the one-pair path's latency."""
    items = device_items(pairs, stream.device)
    eng = engine_for(pairs, device, use_graphs=1)
    if rules:
        eng.set_tile_rules(rules)
    ms = time_batched(eng, items, steps, warmup, stream)
    px = sum(p.P for p in pairs)
    peng = engine_for(pairs[:1], device, use_graphs=1)
    if rules:
        peng.set_tile_rules(rules)
    lat, pv = time_plain(peng, items, stream)
    out = {"workload": pairs[0].name, "pairs": len(pairs),
           "batched": {"value": px / (ms / 1e3) / 1e6, "unit": "Mpix/s", "ms_per_step": ms},
           "plain_graph": plain_line(lat, pv)}
    eng.close()
    peng.close()
    return out


# ---------------------------------------------------------------------------
# serving sweep
# ---------------------------------------------------------------------------

def run_served(pool, device, rules, n_requests, stream):
    """The serving stream over a pool of distinct pairs (request i uses pool
    pair i mod len(pool)) at several Poisson rates, through the
    continuous-batching server and the one-request-per-step server."""
    import torch
    from paper_1501_02565_gb300 import synth
    from paper_1501_02565_gb300.serve import Request, Server, replay
    cfg = dict(max_H=max(p.H for p in pool), max_W=max(p.W for p in pool),
               max_N=max(p.N for p in pool), max_K=100, use_graphs=1)
    # the request submitter and the server loop are Python threads: with the
    # interpreter's default 5 ms switch interval a submission can wait that
    # long for the GIL, and latencies count from the scheduled arrival
    switch = sys.getswitchinterval()
    sys.setswitchinterval(5e-5)
    # capacities: the one-pair path and the batched path on the pool
    items = device_items(pool, stream.device)
    peng = engine_for(pool[:1], device, use_graphs=1)
    if rules:
        peng.set_tile_rules(rules)
    lat, plain_mpix = time_plain(peng, items, stream)
    peng.close()
    beng = engine_for(pool[:32], device, use_graphs=1)
    if rules:
        beng.set_tile_rules(rules)
    ms = time_batched(beng, items[:32], 5, 3, stream)
    beng.close()
    del items
    mean_px = float(np.mean([p.P for p in pool]))
    batched_mpix = sum(p.P for p in pool[:32]) / (ms / 1e3) / 1e6
    c1 = plain_mpix * 1e6 / mean_px                 # requests/s, one at a time
    cb = batched_mpix * 1e6 / mean_px                # requests/s, batched
    rates = [0.5 * c1, 0.9 * c1, 1.5 * c1, 0.7 * cb]
    for p in pool:
        Server.validate(Request(p.C, p.matches, p.K, p.a))
    hostC = [torch.from_numpy(p.C).pin_memory() for p in pool]
    hostM = [torch.from_numpy(p.matches).pin_memory() for p in pool]
    outs = [torch.empty((p.H, p.W, 2), dtype=torch.float32, pin_memory=True) for p in pool]
    sweep = []
    for rate in rates:
        arrivals = synth.serving_requests(n_requests, rate)
        row = {"rate_req_s": rate, "offered_mpix_s": rate * mean_px / 1e6}
        for name, max_batch in (("continuous_batching", 32), ("one_at_a_time", 1)):
            reqs = [Request(hostC[i % len(pool)], hostM[i % len(pool)], pool[i % len(pool)].K,
                            pool[i % len(pool)].a, rid=i, out=outs[i % len(pool)])
                    for i in range(n_requests)]
            srv = Server(device, max_batch=max_batch, **cfg)
            if rules:
                srv.engine.set_tile_rules(rules)
            srv.start()
            warm = [Request(hostC[i], hostM[i], pool[i].K, pool[i].a, rid=-1)
                    for i in range(min(8, len(pool)))]
            for r in warm:
                srv.submit(r, validate=False)
            for r in warm:
                r.wait(timeout=120)
            srv.completed.clear()
            srv.batch_sizes.clear()
            srv.steps = 0
            st = replay(srv, reqs, arrivals, validate=False)
            status = srv.stop()
            st.update({"status": status, "unit": "Mpix/s"})
            row[name] = st
        sweep.append(row)
    sys.setswitchinterval(switch)
    return {"requests_per_rate": n_requests, "distinct_pairs": len(pool),
            "latency_from": "scheduled arrival", "gil_switch_interval_s": 5e-5,
            "sizes": sorted({f"{p.W}x{p.H}" for p in pool}),
            "capacity": {"one_at_a_time_mpix_s": plain_mpix, "batched_mpix_s": batched_mpix,
                         "one_at_a_time_latency_ms_p50": float(np.percentile(lat, 50)),
                         "one_at_a_time_latency_ms_p99": float(np.percentile(lat, 99))},
            "rates": sweep}


# ---------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------

def run_ours(args, rank, world, local_rank):
    import torch
    import torch.distributed as dist
    from paper_1501_02565_gb300.native import EpicInterp
    from paper_1501_02565_gb300.replicas import max_over_ranks, whole_job_rate

    threads = cpu_threads(args)
    extra = not args.no_extra
    # every input, generated before the first GPU call
    jobs = {"head": rank_jobs(HEADLINE_CONFIG, args.batch, rank, world)}
    if rank == 0 and extra:
        jobs["c1"] = [(1, i) for i in range(32)]
        jobs["c2"] = [(2, i) for i in range(32)]
        jobs["c3"] = [(3, i) for i in range(32)]
        if world == 1 and not args.no_serve:
            jobs["c5"] = [(5, i) for i in range(64)]
    flat = [j for v in jobs.values() for j in v]
    made = gen_pairs(flat, threads)
    sets, k = {}, 0
    for name, v in jobs.items():
        sets[name] = made[k:k + len(v)]
        k += len(v)
    pairs = sets["head"]
    B = len(pairs)

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    stream = torch.cuda.Stream(dev)
    items = device_items(pairs, dev)
    step_bytes = sum(it[0].numel() * 4 + it[4].numel() * 4 + it[1].numel() * 4 for it in items)
    # relaxation tiles picked by the autotuner for every size class in use
    tile_rules, tune_report = [], None
    if not args.no_tune:
        from paper_1501_02565_gb300 import tune
        sample = list(pairs)
        for name in ("c1", "c2", "c3"):
            sample += sets.get(name, [])[:16]
        tile_rules, tune_report = tune.autotune(sample, device=local_rank, reps=2, max_batch=16)
        tune_report = {str(k): v for k, v in tune_report.items()}

    def barrier():
        if world > 1:
            dist.barrier()

    # ---- headline: the batch replayed from a captured CUDA graph ----------
    eng = engine_for(pairs, local_rank, use_graphs=1)
    if tile_rules:
        eng.set_tile_rules(tile_rules)
    with torch.cuda.stream(stream):
        for _ in range(max(args.warmup, 3)):
            eng.run_batch(items, stream=stream)
        stream.synchronize()
    eng.sync()
    n_edges = sum(eng.get_edge_count(i) for i in range(B))
    passes = eng.get_passes()
    clocks = ClockSampler(local_rank)
    torch.cuda.synchronize()
    barrier()
    clocks.start()
    with torch.cuda.stream(stream):
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        for _ in range(args.steps):
            eng.run_batch(items, stream=stream)
        ev1.record(stream)
        stream.synchronize()
    barrier()
    ms_total = ev0.elapsed_time(ev1)
    clk = clocks.stop()
    eng.sync()
    ms_total = max_over_ranks(ms_total, dev)
    px_rank = sum(p.P for p in pairs) * args.steps
    value = whole_job_rate(px_rank, world, ms_total / 1e3) / 1e6

    # ---- the same steps with per-kernel CUDA events (plain launches) -------
    eng.enable_stage_timing(True)
    with torch.cuda.stream(stream):
        s0 = torch.cuda.Event(enable_timing=True)
        s1 = torch.cuda.Event(enable_timing=True)
        s0.record(stream)
        for _ in range(args.steps):
            eng.run_batch(items, stream=stream)
        s1.record(stream)
        stream.synchronize()
    stage_ms, n_runs = eng.stage_times()
    eng.enable_stage_timing(False)
    eng.sync()
    ms_plain_launch = s0.elapsed_time(s1) / args.steps

    # ---- end to end through the C ABI with pinned host buffers ------------
    host = []
    for p in pairs:
        host.append((torch.from_numpy(p.C).pin_memory(), torch.from_numpy(p.matches).pin_memory(),
                     p.K, p.a, torch.empty((p.H, p.W, 2), dtype=torch.float32).pin_memory()))
    h2d = sum(h[0].numel() * 4 + h[1].numel() * 4 for h in host)
    d2h = sum(h[4].numel() * 4 for h in host)
    heng = engine_for(pairs, local_rank)
    if tile_rules:
        heng.set_tile_rules(tile_rules)
    heng.run_batch_host(host)
    torch.cuda.synchronize()
    barrier()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        heng.run_batch_host(host)
    t_e2e = time.perf_counter() - t0
    barrier()
    t_e2e = max_over_ranks(t_e2e, dev)
    e2e_blocking = whole_job_rate(px_rank, world, t_e2e) / 1e6
    for _ in range(2):
        heng.submit_batch_host(host)
    heng.sync()
    barrier()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        heng.submit_batch_host(host)
    heng.sync()
    t_e2e = time.perf_counter() - t0
    barrier()
    t_e2e = max_over_ranks(t_e2e, dev)
    e2e_value = whole_job_rate(px_rank, world, t_e2e) / 1e6
    heng.close()
    # sanity: the host result equals the device-resident one
    assert torch.equal(host[0][4], items[0][4].cpu()), "host and device paths differ"
    del host

    # ---- plain one-pair-at-a-time path on the headline pairs --------------
    plain = plain_graph = None
    if extra:
        peng = engine_for(pairs, local_rank)
        if tile_rules:
            peng.set_tile_rules(tile_rules)
        lat, pv = time_plain(peng, items, torch.cuda.current_stream())
        plain = plain_line(lat, pv)
        peng.close()
        geng = engine_for(pairs, local_rank, use_graphs=1)
        if tile_rules:
            geng.set_tile_rules(tile_rules)
        glat, gv = time_plain(geng, items, stream)
        plain_graph = plain_line(glat, gv)
        geng.close()

    # ---- per-configuration lines (configs 1-3) ------------------------------
    configs = None
    if rank == 0 and extra:
        configs = {}
        for name, cfgno in (("c1", 1), ("c2", 2), ("c3", 3)):
            configs[f"config{cfgno}"] = config_line(sets[name], local_rank, tile_rules,
                                                    args.steps, args.warmup, stream)

    # ---- with consistency pruning (Sec. 4.1): two passes per run --------
    pruned = None
    if extra:
        peng = engine_for(pairs, local_rank, prune=1, use_graphs=1)
        if tile_rules:
            peng.set_tile_rules(tile_rules)
        steps_p = max(3, args.steps // 5)
        ms_pruned = time_batched(peng, items, steps_p, 3, stream)
        kept = sum(int(peng.get_pruning(i, p.N)[1].numel()) for i, p in enumerate(pairs))
        pruned = {"value": sum(p.P for p in pairs) / (ms_pruned / 1e3) / 1e6, "unit": "Mpix/s",
                  "ms_per_step": ms_pruned, "steps": steps_p,
                  "kept_frac": kept / sum(p.N for p in pairs),
                  "launches_per_run": peng.launches_per_run(B)}
        peng.close()

    sintel = sets.get("c2") or []
    gradcost = refine = exact = None
    if rank == 0 and extra and sintel:
        from paper_1501_02565_gb300 import synth as _synth
        from paper_1501_02565_gb300.native import gradient_cost
        # ---- image-gradient cost map (Table 2) on 32 Sintel-shaped frames --
        imgs = torch.from_numpy(np.stack([_synth.region_image(p, seed=i) for i, p in
                                          enumerate(sintel)])).to(dev)
        gc_out = torch.empty(imgs.shape[:3], dtype=torch.float32, device=dev)
        for _ in range(3):
            gradient_cost(imgs, 1e-3, out=gc_out)
        torch.cuda.synchronize()
        g0 = torch.cuda.Event(enable_timing=True)
        g1 = torch.cuda.Event(enable_timing=True)
        reps = 20
        cs = torch.cuda.current_stream()
        g0.record(cs)
        for _ in range(reps):
            gradient_cost(imgs, 1e-3, out=gc_out)
        g1.record(cs)
        torch.cuda.synchronize()
        gc_ms = g0.elapsed_time(g1) / reps
        gc_bytes = imgs.numel() * 4 + gc_out.numel() * 4
        gradcost = {"ms_per_launch": gc_ms, "frames": len(sintel),
                    "algorithmic_bytes": gc_bytes,
                    "achieved_gbs": gc_bytes / (gc_ms / 1e3) / 1e9}
        del imgs, gc_out

        # ---- variational refinement (Sec. 4) of one pair ----------------
        p0 = sintel[0]
        it0 = device_items([p0], dev)[0]
        ieng = EpicInterp(local_rank)
        ieng.run_batch([it0])
        ieng.sync()
        approx_lat, _ = time_plain(ieng, [it0] * 8, torch.cuda.current_stream())
        ieng.close()
        im1 = _synth.region_image(p0, seed=0)
        im2 = _synth.second_frame(im1, p0.gt_flow)
        I1t = torch.from_numpy(im1).to(dev)
        I2t = torch.from_numpy(im2).to(dev)
        reng = EpicInterp(local_rank)
        ftmp = it0[4].clone()
        reng.refine(I1t, I2t, ftmp)                      # warm-up, scratch
        times = {}
        for sor_it in (30, 0):
            ftmp.copy_(it0[4])
            r0 = torch.cuda.Event(enable_timing=True)
            r1 = torch.cuda.Event(enable_timing=True)
            r0.record(cs)
            reng.refine(I1t, I2t, ftmp, sor_iterations=sor_it)
            r1.record(cs)
            torch.cuda.synchronize()
            times[sor_it] = r0.elapsed_time(r1)
        ftmp.copy_(it0[4])
        reng.refine(I1t, I2t, ftmp)
        torch.cuda.synchronize()
        gt = torch.from_numpy(p0.gt_flow).to(dev)
        aee0 = float((it0[4] - gt).norm(dim=2).mean())
        aee1 = float((ftmp - gt).norm(dim=2).mean())
        f0 = gt + torch.from_numpy(_synth.smooth_perturbation(p0.H, p0.W, 1.0, seed=3)).to(dev)
        fr = f0.clone()
        reng.refine(I1t, I2t, fr)
        torch.cuda.synchronize()
        vis = torch.from_numpy(_synth.in_frame(p0.gt_flow)).to(dev)
        e0 = (f0 - gt).norm(dim=2)[vis]
        e1 = (fr - gt).norm(dim=2)[vis]
        basin = {"perturbation_rms_px": 1.0, "in_frame_frac": float(vis.float().mean()),
                 "mean_before": float(e0.mean()), "mean_after": float(e1.mean()),
                 "median_before": float(e0.median()), "median_after": float(e1.median())}
        sor_ms = times[30] - times[0]
        sor_bytes = 48.0 * p0.P * 5 * 30   # per SOR iteration and pixel: flow, update, coefficients
        refine = {"pair": f"{p0.W}x{p0.H}", "ms": times[30], "sor_ms": sor_ms,
                  "sor_algorithmic_bytes": sor_bytes,
                  "sor_achieved_gbs": sor_bytes / (sor_ms / 1e3) / 1e9 if sor_ms > 0 else None,
                  "launches": 5 * (3 + 10), "aee_interpolated": aee0, "aee_refined": aee1,
                  "from_perturbed_gt": basin}
        reng.close()
        del I1t, I2t, ftmp

        # ---- exact per-pixel variant (Sec. 5.2, Table 2) on one pair ------
        if not args.no_exact:
            xeng = EpicInterp(local_rank, max_H=p0.H, max_W=p0.W, max_N=p0.N)
            if tile_rules:
                xeng.set_tile_rules(tile_rules)
            exact = {"pair": f"{p0.W}x{p0.H}, N={p0.N}, K={p0.K}"}
            C0, M0 = it0[0], it0[1]
            flows = {}
            for metric in ("geodesic", "euclidean"):
                xeng.exact(C0, M0, p0.K, p0.a, metric=metric)      # warm-up, allocation
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                flows[metric] = xeng.exact(C0, M0, p0.K, p0.a, metric=metric)
                torch.cuda.synchronize()
                exact[f"{metric}_ms"] = 1e3 * (time.perf_counter() - t0)
            exact["approx_ms"] = float(np.median(approx_lat))
            exact["geodesic_over_approx"] = exact["geodesic_ms"] / exact["approx_ms"]
            approx = it0[4]
            exact["aee_approx"] = float((approx - gt).norm(dim=2).mean())
            exact["aee_exact_geodesic"] = float((flows["geodesic"] - gt).norm(dim=2).mean())
            exact["aee_exact_euclidean"] = float((flows["euclidean"] - gt).norm(dim=2).mean())
            exact["mean_approx_to_exact_px"] = float((approx - flows["geodesic"]).norm(dim=2).mean())
            xeng.close()
        del it0

    # ---- served: continuous batching vs one request at a time ------------
    served = None
    if rank == 0 and world == 1 and "c5" in sets:
        served = run_served(sets["c5"], local_rank, tile_rules, args.requests, stream)

    # ---- roofline ----------------------------------------------------------
    peaks, peak_src = measured_peaks()
    hbm = float(peaks["hbm_gbs"])
    if gradcost:
        gradcost["frac_hbm"] = gradcost["achieved_gbs"] / hbm
    stages = {}
    for s in STAGES:
        ms = stage_ms[s] / max(n_runs, 1)
        by = algorithmic_bytes(s, pairs, n_edges)
        gbs = by / (ms / 1e3) / 1e9 if ms > 0 else 0.0
        stages[s] = {"ms_per_launch": ms, "algorithmic_bytes": by, "achieved_gbs": gbs,
                     "frac_hbm": gbs / hbm}
    dom = max(STAGES, key=lambda s: stages[s]["ms_per_launch"])
    traffic, traffic_src = committed_traffic(dom, f"config{HEADLINE_CONFIG}b{B}")
    roofline = {"kernel": dom, "bound": "hbm", "achieved": stages[dom]["achieved_gbs"],
                "peak": hbm, "unit": "GB/s", "frac": stages[dom]["frac_hbm"],
                "traffic": traffic, "peak_source": f"MEASURED_PEAKS.json hbm_gbs ({peak_src})",
                "traffic_source": traffic_src}

    # ---- CPU oracle baseline (rank 0, N = 1 only) ---------------------------
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        sample = reference_sample(pairs, threads)
        t = oracle_pass(sample, threads)
        cpu = {"value": sum(p.P for p in sample) / t / 1e6, "unit": "Mpix/s",
               "cores": min(threads, len(sample)), "kind": "oracle",
               "sample": f"the first {len(sample)} pairs of the headline batch "
                         f"({sum(p.P for p in sample)} pixels), one pair per thread"}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "Mpix/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": ms_total / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "paper_context": {"mpix_s": PAPER_MPIX_S,
                              "what": "0.25 s per 1024x436 pair on one 3.6 GHz CPU core (Sec. 5.4)"},
            "dtype": "f32", "data": "synthetic",
            "config": {"workload": WORKLOAD, "pairs_per_step": B,
                       "pixels_per_step": sum(p.P for p in pairs),
                       "matches_per_step": sum(p.N for p in pairs),
                       "sizes": {s: sum(1 for p in pairs if f"{p.W}x{p.H}" == s)
                                 for s in sorted({f"{p.W}x{p.H}" for p in pairs})},
                       "launch": "batched run replayed from a captured CUDA graph",
                       "parallelism": f"replicas{world}",
                       "tile_rules": [list(r) for r in tile_rules],
                       "l2": f"inputs larger than L2 ({step_bytes / 1e6:.0f} MB of inputs and "
                             f"outputs per step)"},
            "e2e": {"value": e2e_value, "unit": "Mpix/s", "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": d2h, "blocking_value": e2e_blocking,
                    "api": "epic_interp_submit_batch_host per step, one epic_interp_sync"},
            "gpu_launches": eng.launches_per_run(B) * args.steps,
            "roofline": roofline,
            "stages": stages,
            "stages_timed": {"launch": "plain launches, same steps", "steps": n_runs,
                             "ms_per_step": ms_plain_launch},
            "batched_latency_ms": ms_total / args.steps,
            "plain": plain,
            "plain_graph": plain_graph,
            "configs": configs,
            "served": served,
            "pruned": pruned,
            "exact": exact,
            "gradient_cost": gradcost,
            "refine": refine,
            "relax_passes": passes,
            "tune": tune_report,
            "edges_per_step": n_edges,
            "cpu_baseline": cpu,
            "clocks": clk,
        }
        print(json.dumps(line), flush=True)
    eng.close()
    return 0


def main():
    args = parse_args()
    rank = int(os.environ.get("RANK", 0))
    world = int(os.environ.get("WORLD_SIZE", 1))
    local_rank = int(os.environ.get("LOCAL_RANK", 0))
    if args.impl == "reference":
        return run_reference(args, rank, world)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    try:
        return run_ours(args, rank, world, local_rank)
    finally:
        if world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()


if __name__ == "__main__":
    sys.exit(main())
