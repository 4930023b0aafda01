"""A short, fixed launch sequence for kernel profilers.

Runs the batched interpolator on `--batch` Sintel-shaped synthetic pairs
(1024x436, N = 5000, K = 100): `--warmup` runs, then `--runs` runs, then
checks the device status.  Nothing else launches kernels of the library, so
a profiler can skip the warm-up launches by count (6 kernels per run, 12
with --prune) and capture the runs that follow.

  python -m paper_1501_02565_gb300.profile_case --batch 32 --warmup 2 --runs 1
"""

from __future__ import annotations

import argparse
import time


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--batch", type=int, default=32)
    ap.add_argument("--warmup", type=int, default=2)
    ap.add_argument("--runs", type=int, default=1)
    ap.add_argument("--tile", default="64,32,8", help="tile_w,tile_h,apron of the relaxation")
    ap.add_argument("--prune", action="store_true", help="consistency pruning (two passes)")
    args = ap.parse_args(argv)

    import torch
    from . import synth
    from .native import EpicInterp

    tw, th, apron = (int(x) for x in args.tile.split(","))
    pairs = [synth.config_pair(2, i) for i in range(args.batch)]
    dev = torch.device("cuda", 0)
    eng = EpicInterp(0, max_pairs=len(pairs), tile_w=tw, tile_h=th, apron=apron,
                     prune=int(args.prune))
    items = [(torch.from_numpy(p.C).to(dev), torch.from_numpy(p.matches).to(dev), p.K, p.a,
              torch.empty((p.H, p.W, 2), dtype=torch.float32, device=dev)) for p in pairs]
    torch.cuda.synchronize()
    for _ in range(args.warmup):
        eng.run_batch(items)
    eng.sync()
    t0 = time.perf_counter()
    for _ in range(args.runs):
        eng.run_batch(items)
    eng.sync()
    dt = (time.perf_counter() - t0) / max(args.runs, 1)
    print(f"{len(pairs)} pairs, {eng.launches_per_run(len(pairs))} launches per run, "
          f"{dt * 1e3:.2f} ms per run (host clock)")
    eng.close()
    return 0


if __name__ == "__main__":
    raise SystemExit(main())
