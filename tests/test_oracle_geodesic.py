"""Pins for the oracle's assignment map (Sec. 3.4, distance of Eq. 3)."""

import math

import numpy as np
import pytest
import scipy.ndimage as ndi

import oracle
from helpers import brute_assignment, load_golden, random_small_case


@pytest.mark.parametrize("name", ["geodesic_strip.txt", "geodesic_3x3.txt"])
def test_hand_derived_fixtures(name):
    g = load_golden(name)
    D, L = oracle.geodesic(g["C"], g["matches"])
    np.testing.assert_allclose(D, g["D"], rtol=0, atol=1e-12)
    np.testing.assert_array_equal(L, g["L"])


@pytest.mark.parametrize("c", [0.25, 1.0, 3.0])
def test_constant_cost_is_octile_distance(c):
    # On a constant map every axis step costs c and every diagonal c*sqrt2,
    # so the geodesic distance is the octile distance (closed form).
    H, W = 17, 23
    C = np.full((H, W), c, np.float32)
    sx, sy = 7, 5
    m = np.array([[sx, sy, sx, sy]], np.float32)
    D, L = oracle.geodesic(C, m)
    ys, xs = np.mgrid[0:H, 0:W]
    ax, ay = np.abs(xs - sx), np.abs(ys - sy)
    ref = np.float32(c) * (np.maximum(ax, ay) + (math.sqrt(2) - 1) * np.minimum(ax, ay))
    np.testing.assert_allclose(D, ref, rtol=1e-12, atol=1e-12)
    assert (L == 0).all()


@pytest.mark.parametrize("seed", range(6))
def test_matches_bruteforce_per_seed_dijkstra(seed):
    C, m = random_small_case(seed, H=18 + seed, W=21, N=4 + 2 * seed)
    D, L = oracle.geodesic(C, m)
    Db, Lb, tie, _ = brute_assignment(C, m)
    np.testing.assert_allclose(D, Db, rtol=1e-12, atol=1e-12)
    assert (L[~tie] == Lb[~tie]).all()


def test_exact_ties_go_to_smallest_index():
    # Mirror-symmetric cost map and matches: the central column is equidistant
    # from the two matches (identical step sequences), so it must take label 0
    # even though match 1 is listed first in memory order of the pixels.
    H, W = 9, 11
    rng = np.random.default_rng(3)
    half = rng.uniform(0.1, 1.0, size=(H, W // 2 + 1)).astype(np.float32)
    C = np.concatenate([half, half[:, -2::-1]], axis=1)
    assert C.shape == (H, W)
    m = np.array([[W - 2, 4, 0, 0], [1, 4, 0, 0]], np.float32)  # 0 right, 1 left
    D, L = oracle.geodesic(C, m)
    Db, Lb, tie, _ = brute_assignment(C, m)
    np.testing.assert_allclose(D, Db, rtol=1e-12, atol=1e-12)
    assert tie[:, W // 2].all()
    assert (L[:, W // 2] == 0).all()
    assert (L[tie] == 0).all()


def test_duplicate_source_pixels_take_smallest_index():
    C = np.ones((5, 5), np.float32)
    m = np.array([[2, 2, 0, 0], [2, 2, 1, 1], [4, 4, 0, 0]], np.float32)
    D, L = oracle.geodesic(C, m)
    assert L[2, 2] == 0 and D[2, 2] == 0
    assert not (L == 1).any()


def test_invariants_on_polygon_workload():
    from paper_1501_02565_gb300 import synth
    p = synth.config_pair(1, 0)
    D, L = oracle.geodesic(p.C, p.matches)
    xs = p.matches[:, 0].astype(int)
    ys = p.matches[:, 1].astype(int)
    # every match owns its own pixel at distance 0
    assert (D[ys, xs] == 0).all()
    assert (L[ys, xs] == np.arange(p.N)).all()
    assert np.isfinite(D).all() and (L >= 0).all()
    # every cell is one 8-connected component containing its seed
    for m in range(0, p.N, 7):
        comp, n = ndi.label(L == m, structure=np.ones((3, 3)))
        assert n == 1
        assert comp[ys[m], xs[m]] == 1


def test_rejects_match_outside_image():
    C = np.ones((4, 4), np.float32)
    with pytest.raises(RuntimeError):
        oracle.geodesic(C, np.array([[4, 0, 0, 0]], np.float32))
