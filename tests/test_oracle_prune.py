"""Pins for the Nadaraya-Watson interpolation (Eq. 1, Algorithm 1) and the
consistency pruning of Sec. 4.1 ("Pruning of matches": run the NW
interpolation once, drop the matches whose flow is more than 5 px from the
estimate, interpolate with the rest)."""

import numpy as np
import pytest

import oracle


def _grid_matches(H, W, step, flow, jitter_seed=None):
    """Matches on a regular grid (optionally jittered by up to 2 px), every
    one moving by `flow` = (u, v)."""
    ys, xs = np.mgrid[step // 2:H:step, step // 2:W:step]
    xs, ys = xs.ravel().astype(np.float64), ys.ravel().astype(np.float64)
    if jitter_seed is not None:
        rng = np.random.default_rng(jitter_seed)
        xs = np.clip(xs + rng.integers(-2, 3, xs.size), 0, W - 1)
        ys = np.clip(ys + rng.integers(-2, 3, ys.size), 0, H - 1)
    m = np.stack([xs, ys, xs + flow[0], ys + flow[1]], 1).astype(np.float32)
    return m


def _flat(H, W, c=1e-3):
    return np.full((H, W), c, np.float32)


def test_nw_dense_reproduces_a_translation():
    H, W = 40, 56
    m = _grid_matches(H, W, 8, (2.5, -1.25), jitter_seed=3)
    r = oracle.interp(_flat(H, W), m, 25, 1.0, estimator="nw")
    np.testing.assert_allclose(r["flow"][..., 0], 2.5, atol=1e-12)
    np.testing.assert_allclose(r["flow"][..., 1], -1.25, atol=1e-12)


def test_nw_dense_is_constant_per_cell():
    # Sec. 3.4: N_K(p) = N_K(L(p)) and the weights share one factor, so the
    # NW flow is one value per cell: the estimate at the cell's match
    rng = np.random.default_rng(4)
    H, W = 36, 44
    C = rng.uniform(0.01, 1.0, (H, W)).astype(np.float32)
    m = _grid_matches(H, W, 7, (0, 0), jitter_seed=5)
    m[:, 2:] += rng.normal(0, 3, (m.shape[0], 2)).astype(np.float32)
    r = oracle.interp(C, m, 10, 0.7, estimator="nw")
    est = oracle.nw(m, r["idx"], r["dist"], r["count"], 0.7)
    np.testing.assert_allclose(r["flow"], est[r["L"]], atol=1e-12)


def test_consistency_keeps_everything_on_a_translation():
    H, W = 40, 56
    m = _grid_matches(H, W, 8, (-4.0, 6.0), jitter_seed=6)
    keep, dev, _ = oracle.consistency(_flat(H, W), m, 1.0, threshold=1e-9)
    assert keep.all()
    assert dev.max() < 1e-12


def test_planted_outliers_are_exactly_the_ones_removed():
    # a translation with isolated matches pushed 20 px off: with 25
    # neighbours of nearly equal weight (flat cost), an outlier sits about
    # 20 (1 - 1/25) px from its estimate and an inlier next to it under
    # 20 / 25 px from its own
    H, W = 64, 96
    m = _grid_matches(H, W, 8, (3.0, 1.0))
    out = np.array([5, 30, 61, 88])
    m[out, 2] += 12.0
    m[out, 3] += 16.0          # offset (12, 16): 20 px
    keep, dev, _ = oracle.consistency(_flat(H, W), m, 1.0, threshold=5.0, K_nw=25)
    assert np.flatnonzero(~keep).tolist() == out.tolist()
    assert (dev[out] > 15).all() and (np.delete(dev, out) < 2).all()
    # the pruned interpolation no longer sees them: LA reproduces the
    # translation everywhere (it reproduces any affine field exactly)
    r = oracle.interp_pruned(_flat(H, W), m, 50, 1.0)
    assert r["kept_index"].tolist() == np.flatnonzero(keep).tolist()
    np.testing.assert_allclose(r["flow"][..., 0], 3.0, atol=1e-9)
    np.testing.assert_allclose(r["flow"][..., 1], 1.0, atol=1e-9)
    # without pruning the outliers leak into the field
    r0 = oracle.interp(_flat(H, W), m, 50, 1.0)
    assert np.abs(r0["flow"][..., 0] - 3.0).max() > 1.0


def test_deviation_is_euclidean_and_scales_with_the_offset():
    H, W = 48, 64
    base = _grid_matches(H, W, 8, (0.0, 0.0))
    devs = []
    for s in (1.0, 2.0):
        m = base.copy()
        m[10, 2] += 3 * s
        m[10, 3] -= 4 * s
        _, dev, _ = oracle.consistency(_flat(H, W), m, 1.0, K_nw=25)
        devs.append(dev[10])
    # the estimate is linear in the flows: doubling the offset doubles it
    assert devs[1] == pytest.approx(2 * devs[0], rel=1e-12)
    assert 5 * (1 - 1 / 20) < devs[0] < 5


def test_threshold_is_inclusive():
    # "over 5 pixels" is removed: a deviation equal to the threshold stays
    H, W = 40, 56
    m = _grid_matches(H, W, 8, (0.0, 0.0))
    m[7, 2] += 9.0
    _, dev, _ = oracle.consistency(_flat(H, W), m, 1.0)
    d = float(dev[7])
    keep_at, _, _ = oracle.consistency(_flat(H, W), m, 1.0, threshold=d)
    keep_below, _, _ = oracle.consistency(_flat(H, W), m, 1.0,
                                          threshold=np.nextafter(d, 0.0))
    assert keep_at[7] and not keep_below[7]


def test_nothing_consistent_keeps_all_matches():
    # two matches with opposite 30 px flows: each is about 15 px from the
    # average of the two, so neither passes and both are kept
    H, W = 20, 40
    m = np.array([[5, 10, 35, 10], [30, 10, 0, 10]], np.float32)
    r = oracle.interp_pruned(_flat(H, W), m, 2, 1.0, K_nw=2)
    assert not r["keep"].any()
    assert r["kept_index"].tolist() == [0, 1]
    np.testing.assert_array_equal(r["flow"], oracle.interp(_flat(H, W), m, 2, 1.0)["flow"])
