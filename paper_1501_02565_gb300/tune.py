"""Autotuner for the relaxation's tile shape and sweep schedule.

The tile (width x height, plus the apron of context used in the first pass)
and the sweep schedule (lines cut into segments for every thread, or whole
lines per thread) change only speed, never results: every tiling and
schedule reaches the same fixed point of the relaxation.  Which is fastest
depends on the frame size (how many tiles there are to fill the GPU), the
batch size and the match density, so the tuner times candidates on sample
pairs of each size class with the library's own per-stage CUDA-event
timing and installs the winners as tile rules
(``epic_interp_set_tile_rules``).  Results are cached in a JSON file keyed
by GPU name and size class.
"""

from __future__ import annotations

import json
import os

# (tile_w, tile_h, apron, sweep).  sweep 2: the row-closure passes on warp
# tiles of 64 x tile_h (the interpolator's default relaxation); the library
# uses them only when every rule asks for them, so a rule set is tuned from
# one family at a time.
CANDIDATES = ((64, 32, 0, 2), (64, 16, 0, 2), (64, 12, 0, 2), (64, 8, 0, 2))
# sweep 0 / 1: the sweep schedules of the tiled relaxation with an apron
# (region = tile + 2 apron within shared memory at 256 threads per CTA)
SWEEP_CANDIDATES = (
    (64, 32, 4, 0), (32, 32, 4, 0), (64, 32, 0, 0), (64, 32, 8, 0), (48, 48, 8, 0),
    (64, 64, 8, 0), (96, 32, 4, 0), (128, 32, 4, 0), (32, 16, 2, 0), (128, 64, 8, 0),
    (64, 32, 8, 1), (48, 48, 8, 1), (32, 32, 4, 1),
)

# size classes: upper pixel bounds (a frame uses the first class that holds it)
CLASS_BOUNDS = (1 << 16, 1 << 18, 1 << 19, 1 << 20, 1 << 21, 1 << 23)


def size_class(pixels: int) -> int:
    """Upper pixel bound of the class holding a frame of `pixels` pixels."""
    for b in CLASS_BOUNDS:
        if pixels <= b:
            return b
    return 1 << 62


def group_by_class(pairs):
    groups = {}
    for p in pairs:
        groups.setdefault(size_class(p.H * p.W), []).append(p)
    return dict(sorted(groups.items()))


# the bound given to the last rule: every larger frame uses it too, so the
# handle's configured tile never applies (and a captured launch sequence is
# sized for the tuned tiles alone)
ALL_SIZES = 1 << 62


def rules_from_choice(choice):
    """{class bound: (tw, th, apron[, sweep])} -> sorted rule list for the
    library; the largest class's rule also covers every larger frame."""
    bounds = sorted(choice)
    return [(ALL_SIZES if i == len(bounds) - 1 else b, *choice[b]) for i, b in enumerate(bounds)]


def time_candidate(pairs, tile, device=0, reps=3, warmup=2):
    """Mean milliseconds per run of the relaxation + edge stages (the two the
    tile affects) on one batch of `pairs`."""
    import torch
    from .native import EpicInterp
    tw, th, ap = tile[:3]
    sw = tile[3] if len(tile) > 3 else 0
    eng = EpicInterp(device, tile_w=tw, tile_h=th, apron=ap, sweep=sw, max_pairs=len(pairs))
    try:
        dev = torch.device("cuda", device)
        items = [(torch.from_numpy(p.C).to(dev), torch.from_numpy(p.matches).to(dev), p.K, p.a,
                  torch.empty((p.H, p.W, 2), dtype=torch.float32, device=dev)) for p in pairs]
        for _ in range(warmup):
            eng.run_batch(items)
        eng.sync()
        eng.enable_stage_timing(True)
        for _ in range(reps):
            eng.run_batch(items)
        st, n = eng.stage_times()
        eng.sync()
        return (st["relax"] + st["edges"]) / max(n, 1)
    finally:
        eng.close()


def autotune(pairs, device=0, candidates=CANDIDATES, reps=3, max_batch=32, log=None):
    """Pick the fastest tile per size class; returns (rules, report)."""
    choice, report = {}, {}
    for bound, group in group_by_class(pairs).items():
        sample = group[:max_batch]
        times = {}
        for tile in candidates:
            try:
                times[tile] = time_candidate(sample, tile, device, reps)
            except Exception as exc:  # a shape that does not fit this GPU
                if log:
                    log(f"tile {tile} skipped: {exc}")
        best = min(times, key=times.get)
        choice[bound] = best
        report[bound] = {"best": list(best),
                         "ms": {f"{t[0]}x{t[1]}+{t[2]}" + ("w" if len(t) > 3 and t[3] else ""): v
                                for t, v in times.items()},
                         "pairs": len(sample)}
    return rules_from_choice(choice), report


def save_rules(path, rules, gpu_name, report=None):
    data = {}
    if os.path.exists(path):
        with open(path) as f:
            data = json.load(f)
    data[gpu_name] = {"rules": [list(r) for r in rules], "report": report or {}}
    tmp = path + ".tmp"
    with open(tmp, "w") as f:
        json.dump(data, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def load_rules(path, gpu_name):
    if not os.path.exists(path):
        return None
    with open(path) as f:
        data = json.load(f)
    entry = data.get(gpu_name)
    return [tuple(r) for r in entry["rules"]] if entry else None
