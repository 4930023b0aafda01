"""Tile autotuner: size classes, rule construction and the JSON cache (CPU),
and on the GPU that tuned rules change speed only, never results."""

import numpy as np
import pytest

from paper_1501_02565_gb300 import synth, tune


def test_size_classes_are_monotone_and_cover_everything():
    sizes = [1, 5000, 1 << 16, (1 << 16) + 1, 446464, 1 << 21, 1 << 30]
    cls = [tune.size_class(s) for s in sizes]
    assert all(c >= s for c, s in zip(cls, sizes))
    assert cls == sorted(cls)
    assert tune.size_class(1 << 16) == 1 << 16


def test_rules_are_sorted_by_class():
    rules = tune.rules_from_choice({1 << 20: (64, 32, 4), 1 << 16: (32, 16, 2)})
    # the largest class's rule covers every larger frame as well
    assert rules == [(1 << 16, 32, 16, 2), (tune.ALL_SIZES, 64, 32, 4)]


def test_cache_round_trip(tmp_path):
    path = str(tmp_path / "tiles.json")
    rules = [(1 << 19, 64, 32, 4)]
    tune.save_rules(path, rules, "GPU A", {"x": 1})
    tune.save_rules(path, [(1 << 20, 32, 32, 0)], "GPU B")
    assert tune.load_rules(path, "GPU A") == rules
    assert tune.load_rules(path, "GPU B") == [(1 << 20, 32, 32, 0)]
    assert tune.load_rules(path, "GPU C") is None


def test_candidates_are_valid_tiles():
    # warp tiles: 64 columns, 1..32 rows, no apron
    for tw, th, ap, sw in tune.CANDIDATES:
        assert sw == 2 and tw == 64 and 1 <= th <= 32 and ap == 0
    for tw, th, ap, sw in tune.SWEEP_CANDIDATES:
        assert 8 <= tw <= 256 and 8 <= th <= 256 and 0 <= ap <= 64
        assert ap + 1 <= min(tw, th)
        assert sw in (0, 1)
    assert any(c[3] == 1 for c in tune.SWEEP_CANDIDATES)
    assert any(c[3] == 0 for c in tune.SWEEP_CANDIDATES)


@pytest.mark.gpu
def test_tuned_rules_leave_results_unchanged():
    import torch
    from paper_1501_02565_gb300.native import EpicInterp
    pairs = [synth.config_pair(1, i) for i in range(3)] + [synth.config_pair(2, 0)]
    rules, report = tune.autotune(pairs, candidates=tune.CANDIDATES[:4], reps=1)
    print("\n[tune]", rules, report)
    assert len(rules) == 2
    eng_t = EpicInterp(0)
    eng_t.set_tile_rules(rules)
    eng_d = EpicInterp(0)
    for p in pairs:
        C = torch.from_numpy(p.C).cuda()
        M = torch.from_numpy(p.matches).cuda()
        ft = eng_t.run(C, M, p.K, p.a)
        fd = eng_d.run(C, M, p.K, p.a)
        eng_t.sync()
        eng_d.sync()
        assert torch.equal(ft, fd)
    with pytest.raises(Exception):
        eng_t.set_tile_rules([(100, 4, 4, 0)])   # tile side below 8
    eng_t.close()
    eng_d.close()
