"""Nadaraya-Watson interpolation and consistency pruning on the GPU vs the
FP64 oracle (Eq. 1, Algorithm 1, Sec. 4.1 "Pruning of matches").

A pruned run is two passes of the same kernels with a compaction between
them, all on the device.  Its checks:
  * the keep flags equal the oracle's consistency check run on the GPU's
    first-pass labelling, except for matches whose deviation is within
    KEEP_TOL of the threshold or whose K-th neighbour nearly ties;
  * the second pass is the plain interpolator on the kept matches: its flow,
    labels and models equal, bit for bit, a plain run on those matches;
  * NW interpolation (estimator = 1) meets the flow tolerance of parity.py.
"""

import numpy as np
import pytest

import oracle
from paper_1501_02565_gb300 import synth
from parity import full_parity, knn_near_ties, oracle_on_labels, run_gpu

pytestmark = pytest.mark.gpu

THR = 5.0
K_NW = 25
KEEP_TOL = 1e-3   # px: GPU NW estimates carry ~1e-5 px error


def _engine(**cfg):
    from paper_1501_02565_gb300.native import EpicInterp
    cfg.setdefault("keep_intermediates", 1)
    return EpicInterp(0, **cfg)


def _pruned_run(p, eng=None, **cfg):
    import torch
    own = eng is None
    if own:
        eng = _engine(prune=1, prune_threshold=THR, prune_K=K_NW, **cfg)
    C = torch.from_numpy(p.C).cuda()
    M = torch.from_numpy(p.matches).cuda()
    flow = eng.run(C, M, p.K, p.a)
    eng.sync()
    keep, kept = eng.get_pruning(0, p.N)
    L, D = eng.get_labels(0, p.H, p.W)
    out = dict(flow=flow.cpu().numpy(), keep=keep.cpu().numpy().astype(bool),
               kept=kept.cpu().numpy(), L=L.cpu().numpy(), D=D.cpu().numpy())
    models, _ = eng.get_models(0, len(out["kept"]))
    out["models"] = models.cpu().numpy()
    if own:
        eng.close()
    return out


def _check_keep_flags(p, g):
    """GPU keep flags vs the oracle's check on the GPU's first-pass labels."""
    first = run_gpu(p, K=K_NW, estimator=1)       # the first pass, alone
    ref = oracle.interp(p.C, p.matches, K_NW, p.a, estimator="nw")
    refb = oracle_on_labels(p.C, p.matches, K_NW, p.a, ref["D"], first["L"],
                            estimator="nw")
    own = p.matches[:, 2:].astype(np.float64) - p.matches[:, :2]
    dev = np.hypot(*(refb["model"][:, :2] - own).T)
    keep_ref = dev <= THR
    excused = (np.abs(dev - THR) <= KEEP_TOL) | knn_near_ties(p.matches, refb)
    diff = (g["keep"] != keep_ref) & ~excused
    assert not diff.any(), f"{diff.sum()} keep flags differ: {np.flatnonzero(diff)[:10]}"
    return keep_ref, int(excused.sum())


def test_nw_interpolation_parity():
    p = synth.config_pair(1, 0)
    g, ref, rep = full_parity(p, K=K_NW, estimator="nw")
    print("\n[nw] " + " ".join(f"{k}={v}" for k, v in rep.items()))
    assert (g["fallback"] == 1).all()
    # constant flow per cell (Algorithm 1, step 8)
    assert (g["models"][:, 2:6] == 0).all()


@pytest.mark.parametrize("index", [0, 1])
def test_keep_flags_match_oracle(index):
    p = synth.config_pair(1, index)
    g = _pruned_run(p)
    keep_ref, n_exc = _check_keep_flags(p, g)
    print(f"\n[keep{index}] kept={g['keep'].sum()}/{p.N} excused={n_exc}")
    # the synthetic outliers (5 %) go, and so do some matches at motion
    # boundaries, where the NW average mixes two motions
    assert 0.7 * p.N < g["keep"].sum() < p.N
    expect = np.flatnonzero(g["keep"]) if g["keep"].any() else np.arange(p.N)
    assert np.array_equal(g["kept"], expect)


def test_pruned_run_is_plain_run_on_kept_matches():
    p = synth.config_pair(1, 2)
    g = _pruned_run(p)
    q = synth.Pair(p.H, p.W, p.C, np.ascontiguousarray(p.matches[g["kept"]]), p.gt_flow,
                   p.K, p.a, p.name)
    plain = run_gpu(q)
    assert np.array_equal(g["L"], plain["L"])
    assert np.array_equal(g["D"], plain["D"])
    assert np.array_equal(g["flow"], plain["flow"])
    assert np.array_equal(g["models"], plain["models"])


def test_pruned_flow_vs_oracle():
    # end to end: the oracle's pruned interpolation on the GPU's kept set
    # (equal to the oracle's own set up to the excused flags above)
    p = synth.config_pair(1, 3)
    g = _pruned_run(p)
    q = (p.C, np.ascontiguousarray(p.matches[g["kept"]]))
    _, _, rep = full_parity(q, K=p.K, a=p.a)
    print("\n[pruned] " + " ".join(f"{k}={v}" for k, v in rep.items()))
    # the planted outliers (flow more than 10 px off the ground truth at
    # their source pixel) are what the check is for: most of them go
    xs = np.floor(p.matches[:, 0] + 0.5).astype(int)
    ys = np.floor(p.matches[:, 1] + 0.5).astype(int)
    off = np.hypot(*(p.matches[:, 2:] - p.matches[:, :2] - p.gt_flow[ys, xs]).T)
    outlier = off > 10
    recall = float((~g["keep"][outlier]).mean())
    plain = run_gpu(p)
    err_p = np.hypot(*(g["flow"] - p.gt_flow).transpose(2, 0, 1)).mean()
    err_0 = np.hypot(*(plain["flow"] - p.gt_flow).transpose(2, 0, 1)).mean()
    print(f"[pruned] outliers {outlier.sum()} removed {recall:.2f}; "
          f"AEE to ground truth {err_0:.3f} (all) -> {err_p:.3f} (pruned)")
    assert recall >= 0.7


def test_nothing_consistent_keeps_all():
    C = np.full((20, 40), 1e-3, np.float32)
    M = np.array([[5, 10, 35, 10], [30, 10, 0, 10]], np.float32)
    p = synth.Pair(20, 40, C, M, np.zeros((20, 40, 2), np.float32), 2, 1.0, "two")
    import torch
    eng = _engine(prune=1, prune_threshold=THR, prune_K=2)
    flow = eng.run(torch.from_numpy(C).cuda(), torch.from_numpy(M).cuda(), 2, 1.0)
    eng.sync()
    keep, kept = eng.get_pruning(0, 2)
    assert keep.cpu().tolist() == [0, 0]
    assert kept.cpu().tolist() == [0, 1]
    ref = oracle.interp_pruned(C, M, 2, 1.0, K_nw=2)
    np.testing.assert_allclose(flow.cpu().numpy(), ref["flow"], atol=1e-4)
    eng.close()


def test_pruned_batch_and_graph_replay_match_single_runs():
    import torch
    pairs = [synth.config_pair(1, i) for i in range(3)]
    singles = [_pruned_run(p)["flow"] for p in pairs]
    eng = _engine(prune=1, prune_threshold=THR, prune_K=K_NW, use_graphs=1, max_pairs=3,
                  max_H=128, max_W=256, max_N=600, max_K=32)
    s = torch.cuda.Stream()
    dev = [(torch.from_numpy(p.C).cuda(), torch.from_numpy(p.matches).cuda(), p.K, p.a,
            torch.empty((p.H, p.W, 2), dtype=torch.float32, device="cuda")) for p in pairs]
    torch.cuda.synchronize()
    for rep in range(3):  # capture, then replays
        with torch.cuda.stream(s):
            eng.run_batch(dev, stream=s)
        s.synchronize()
        eng.sync()
        for i in range(3):
            assert np.array_equal(dev[i][4].cpu().numpy(), singles[i]), (rep, i)
        assert eng.launches_per_run(3) == 20
    eng.close()
