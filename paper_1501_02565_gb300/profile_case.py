"""A short, fixed launch sequence for kernel profilers.

--what interp (default): the batched interpolator on `--batch` synthetic
pairs of `--config` (2: Sintel-shaped 1024x436, N = 5000, K = 100; 4: the
mixed-size batch): `--warmup` runs, then `--runs` runs, then the device
status is checked.  10 kernels per
run (20 with --prune).
--what gradcost: the image-gradient cost map of `--batch` synthetic frames,
one launch per run.
--what refine: the variational refinement of the first pair's interpolated
flow (one interpolation run first), 5 x (3 + 10) launches per run.

Nothing else launches kernels of the library, so a profiler can skip the
warm-up launches by count and capture the runs that follow.

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
    ap.add_argument("--tile", default="64,16,0", help="tile_w,tile_h,apron of the relaxation")
    ap.add_argument("--sweep", type=int, default=2, help="relaxation schedule (0, 1, 2)")
    ap.add_argument("--config", type=int, default=2,
                    help="2: Sintel-shaped pairs; 4: the mixed-size batch")
    ap.add_argument("--prune", action="store_true", help="consistency pruning (two passes)")
    ap.add_argument("--what", default="interp", choices=("interp", "gradcost", "refine"))
    args = ap.parse_args(argv)
    if args.what != "interp":
        return _other(args)

    import torch
    from . import synth
    from .native import EpicInterp

    tw, th, apron = (int(x) for x in args.tile.split(","))
    pairs = [synth.config_pair(args.config, i) for i in range(args.batch)]
    dev = torch.device("cuda", 0)
    eng = EpicInterp(0, max_pairs=len(pairs), tile_w=tw, tile_h=th, apron=apron,
                     sweep=args.sweep, prune=int(args.prune),
                     max_H=max(p.H for p in pairs), max_W=max(p.W for p in pairs),
                     max_N=max(p.N for p in pairs), max_K=max(p.K for p in pairs))
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


def _other(args):
    import numpy as np
    import torch
    from . import synth
    from .native import EpicInterp, gradient_cost
    dev = torch.device("cuda", 0)
    if args.what == "gradcost":
        pairs = [synth.config_pair(2, i) for i in range(args.batch)]
        imgs = torch.from_numpy(np.stack([synth.region_image(p, seed=i)
                                          for i, p in enumerate(pairs)])).to(dev)
        out = torch.empty(imgs.shape[:3], dtype=torch.float32, device=dev)
        for _ in range(args.warmup + args.runs):
            gradient_cost(imgs, 1e-3, out=out)
        torch.cuda.synchronize()
        print(f"{args.batch} frames, 1 launch per run")
        return 0
    p = synth.config_pair(2, 0)
    eng = EpicInterp(0)
    flow0 = eng.run(torch.from_numpy(p.C).to(dev), torch.from_numpy(p.matches).to(dev), p.K, p.a)
    eng.sync()
    im1 = synth.region_image(p, seed=0)
    I1 = torch.from_numpy(im1).to(dev)
    I2 = torch.from_numpy(synth.second_frame(im1, p.gt_flow)).to(dev)
    f = flow0.clone()
    for _ in range(args.warmup + args.runs):
        f.copy_(flow0)
        eng.refine(I1, I2, f)
    torch.cuda.synchronize()
    eng.close()
    print("1 pair, 7 interpolation launches, then 5 x (3 + 10) refinement launches per run")
    return 0


if __name__ == "__main__":
    raise SystemExit(main())
