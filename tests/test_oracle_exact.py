"""Pins for the exact variant of Sec. 5.2 (Table 2, "Geodesic (exact)" and
"Euclidean"): distances from every pixel to every match, the K nearest per
pixel and a fit per pixel."""

import numpy as np
import pytest
from scipy.spatial.distance import cdist

import oracle
from helpers import lstsq_model, random_small_case


def test_exact_geodesic_on_constant_cost_is_octile():
    # constant C: the cheapest 8-connected path has max(dx,dy)-min(dx,dy)
    # axis steps and min(dx,dy) diagonal steps, each costing C times its length
    H, W, c = 13, 17, 0.4
    C = np.full((H, W), c, np.float32)
    m = np.array([[3, 4, 0, 0], [15, 11, 0, 0], [8, 0, 0, 0]], np.float32)
    D = oracle.exact_distances(C, m)
    ys, xs = np.mgrid[0:H, 0:W]
    for i in range(3):
        dx, dy = np.abs(xs - m[i, 0]), np.abs(ys - m[i, 1])
        ref = np.float32(c) * (np.maximum(dx, dy) - np.minimum(dx, dy) + np.sqrt(2) * np.minimum(dx, dy))
        np.testing.assert_allclose(D[i], ref, rtol=1e-12)


def test_exact_euclidean_matches_cdist():
    C, m = random_small_case(71, H=9, W=11, N=6)
    D = oracle.exact_distances(C, m, metric="euclidean")
    pix = np.stack(np.mgrid[0:9, 0:11][::-1], -1).reshape(-1, 2)
    ref = cdist(np.floor(m[:, :2].astype(np.float64) + 0.5), pix).reshape(6, 9, 11)
    np.testing.assert_allclose(D, ref, rtol=1e-14, atol=1e-14)


@pytest.mark.parametrize("weight_squared", [True, False])
def test_fit_points_equals_independent_lstsq(weight_squared):
    rng = np.random.default_rng(5)
    C, m = random_small_case(72, H=16, W=20, N=14)
    centres = rng.integers(0, 16, (9, 2)).astype(np.float64)
    idx = np.stack([rng.choice(14, 8, replace=False) for _ in range(9)]).astype(np.int32)
    dist = rng.uniform(0, 2, (9, 8))
    model, fb, _ = oracle.fit_points(centres, m, idx, dist, np.full(9, 8, np.int32), 0.8,
                                     weight_squared)
    assert not fb.any()
    for i in range(9):
        # lstsq_model centres at match row `i` of its first argument: put the
        # centre there as a pseudo-match
        mm = np.concatenate([m, [[centres[i, 0], centres[i, 1], 0, 0]]]).astype(np.float32)
        ref = lstsq_model(mm, len(m), idx[i], dist[i], 0.8, weight_squared)
        np.testing.assert_allclose(model[i], ref, rtol=1e-8, atol=1e-8)


def test_exact_recovers_a_global_affine_field():
    C, m = random_small_case(73, H=18, W=22, N=16, c_lo=0.05, c_hi=1.0)
    A = np.array([[1.02, -0.03], [0.04, 0.97]])
    t = np.array([2.5, -1.0])
    m[:, 2:] = (m[:, :2].astype(np.float64) @ A.T + t).astype(np.float32)
    for metric in ("geodesic", "euclidean"):
        # a small kernel coefficient keeps the 8 weights comparable, so no
        # fit is degenerate (a degenerate one falls back to NW)
        r = oracle.interp_exact(C, m, 8, 0.05, metric=metric)
        assert not r["fallback"].any()
        ys, xs = np.mgrid[0:18, 0:22]
        p = np.stack([xs, ys], -1).astype(np.float64)
        # targets are float32-rounded: compare at that precision
        np.testing.assert_allclose(r["flow"], p @ A.T + t - p, atol=2e-4)


def test_exact_neighbour_distances_bound_the_approximation():
    # Eq. 4: D~(p, p_n) = D(p) + d_G(L(p), n) >= D_G(p, p_n) for every n, so
    # the k-th exact distance at a pixel never exceeds the k-th approximate one
    C, m = random_small_case(74, H=20, W=24, N=12)
    K = 6
    ex = oracle.interp_exact(C, m, K, 1.0)
    ap = oracle.interp(C, m, K, 1.0)
    L = ap["L"].ravel()
    approx = ap["D"].ravel()[:, None] + ap["dist"][L]
    assert (ex["dist"] <= approx + 1e-9).all()
    assert (ex["dist"][:, 0] <= ap["D"].ravel() + 1e-12).all()


def test_exact_one_neighbour_nw_is_the_voronoi_flow():
    # K = 1: both the exact and the approximate interpolators give every
    # pixel the flow of its nearest match, i.e. of its Voronoi cell L(p)
    C, m = random_small_case(75, H=20, W=24, N=12)
    ex = oracle.interp_exact(C, m, 1, 1.0, estimator="nw")
    ap = oracle.interp(C, m, 1, 1.0, estimator="nw")
    np.testing.assert_array_equal(ex["idx"][:, 0], ap["L"].ravel())
    np.testing.assert_allclose(ex["flow"], ap["flow"], atol=1e-12)
