"""Pins for the per-match LA fit (Eq. 2 restricted to N_K, Sec. 3.2/3.4) and
the Nadaraya-Watson estimate (Eq. 1)."""

import numpy as np
import pytest

import oracle
from helpers import lstsq_model


def _random_neighbourhoods(seed, N=50, K=12):
    rng = np.random.default_rng(seed)
    m = np.zeros((N, 4), np.float32)
    m[:, 0] = rng.integers(0, 200, N)
    m[:, 1] = rng.integers(0, 120, N)
    m[:, 2] = m[:, 0] + rng.normal(0, 20, N)
    m[:, 3] = m[:, 1] + rng.normal(0, 20, N)
    idx = np.zeros((N, K), np.int32)
    dist = np.zeros((N, K))
    for i in range(N):
        others = rng.choice(np.delete(np.arange(N), i), K - 1, replace=False)
        idx[i] = np.concatenate([[i], others])
        dist[i] = np.concatenate([[0.0], np.sort(rng.uniform(0, 3, K - 1))])
    count = np.full(N, K, np.int32)
    return m, idx, dist, count


@pytest.mark.parametrize("weight_squared", [True, False])
@pytest.mark.parametrize("a", [0.5, 1.0, 2.0])
def test_fit_equals_independent_weighted_lstsq(weight_squared, a):
    m, idx, dist, count = _random_neighbourhoods(11)
    model, fb, _ = oracle.fit(m, idx, dist, count, a, weight_squared)
    assert not fb.any()
    for i in range(m.shape[0]):
        ref = lstsq_model(m, i, idx[i], dist[i], a, weight_squared)
        np.testing.assert_allclose(model[i], ref, rtol=1e-9, atol=1e-9)


def test_global_affine_is_recovered_exactly():
    # Noise-free matches of one affine map p' = A p + t: every weighted fit
    # must return B = A - I and c = A p_m + t - p_m whatever the weights.
    rng = np.random.default_rng(5)
    A = np.array([[1.03, -0.02], [0.04, 0.97]])
    t = np.array([7.5, -3.25])
    m, idx, dist, count = _random_neighbourhoods(12)
    p = m[:, :2].astype(np.float64)
    q = p @ A.T + t
    m[:, 2:] = q.astype(np.float32)
    model, fb, _ = oracle.fit(m, idx, dist, count, 1.0)
    qf = m[:, 2:].astype(np.float64)  # float32-rounded targets
    for i in range(m.shape[0]):
        nb = idx[i]
        # exact solution for the float32 targets differs from A, t by the
        # rounding of q; compare with the map fitted to these exact targets
        X = np.stack([p[nb, 0] - p[i, 0], p[nb, 1] - p[i, 1], np.ones(len(nb))], 1)
        bu = np.linalg.lstsq(X, qf[nb, 0] - p[nb, 0], rcond=None)[0]
        np.testing.assert_allclose(model[i, [2, 3, 0]], bu, atol=2e-5)
        np.testing.assert_allclose(model[i, 2:], (A - np.eye(2)).ravel(), atol=1e-5)
        np.testing.assert_allclose(model[i, :2], q[i] - p[i], atol=1e-4)


def test_scaling_all_weights_leaves_model_unchanged():
    # Sec. 3.4: the LA estimator is invariant to multiplying every weight by
    # one constant, which is what adding a constant to every distance does.
    m, idx, dist, count = _random_neighbourhoods(13)
    a = 1.0
    m0, _, _ = oracle.fit(m, idx, dist, count, a)
    m1, _, _ = oracle.fit(m, idx, dist + 2.5, count, a)
    np.testing.assert_allclose(m0, m1, rtol=1e-9, atol=1e-9)


def test_degenerate_neighbourhood_falls_back_to_nadaraya_watson():
    # all neighbours on one line: the normal matrix is singular
    N = 6
    m = np.zeros((N, 4), np.float32)
    m[:, 0] = np.arange(N) * 3
    m[:, 1] = 10
    m[:, 2] = m[:, 0] + np.arange(N)
    m[:, 3] = m[:, 1] - 2 * np.arange(N)
    idx = np.tile(np.arange(N, dtype=np.int32), (N, 1))
    for i in range(N):
        idx[i] = np.concatenate([[i], np.delete(np.arange(N), i)])
    dist = np.tile(np.linspace(0, 1, N), (N, 1))
    count = np.full(N, N, np.int32)
    model, fb, dr = oracle.fit(m, idx, dist, count, 1.0)
    assert fb.all()
    k = np.exp(-dist[0])
    for i in range(N):
        # neighbour n has flow (n, -2n): the fallback is the k-weighted mean
        # flow, held constant over the cell (B = 0)
        n = idx[i].astype(np.float64)
        ref = [(k * n).sum() / k.sum(), (k * -2 * n).sum() / k.sum()]
        np.testing.assert_allclose(model[i, :2], ref, rtol=1e-12, atol=1e-12)
        assert (model[i, 2:] == 0).all()


def test_fewer_than_three_neighbours_falls_back():
    # flows (1, 1) and (4, 4); match 0 sees itself (k = 1) and match 1
    # (k = e^-1): estimate (1 + 4/e) / (1 + 1/e) by hand
    m = np.array([[0, 0, 1, 1], [5, 5, 9, 9]], np.float32)
    idx = np.array([[0, 1], [1, 0]], np.int32)
    dist = np.array([[0, 1.0], [0, 1.0]])
    model, fb, _ = oracle.fit(m, idx, dist, np.array([2, 2], np.int32), 1.0)
    assert fb.all()
    e = np.e
    np.testing.assert_allclose(model[0, :2], [(1 + 4 / e) / (1 + 1 / e)] * 2, rtol=1e-14)
    np.testing.assert_allclose(model[1, :2], [(4 + 1 / e) / (1 + 1 / e)] * 2, rtol=1e-14)


def test_nadaraya_watson_reproduces_a_translation():
    # Eq. 1 is a weighted mean: every neighbour moving by the same (u, v)
    # gives exactly (u, v), whatever the weights and wherever the
    # neighbours sit (a position average would be pulled towards the
    # neighbours' centroid instead)
    m, idx, dist, count = _random_neighbourhoods(15)
    m[:, 2] = m[:, 0] + 3.25
    m[:, 3] = m[:, 1] - 7.5
    for a in (0.3, 1.0, 4.0):
        out = oracle.nw(m, idx, dist, count, a)
        np.testing.assert_allclose(out, np.tile([3.25, -7.5], (m.shape[0], 1)), atol=1e-12)


def test_nadaraya_watson_single_neighbour_is_own_flow():
    m, idx, dist, count = _random_neighbourhoods(16)
    out = oracle.nw(m, idx, dist, np.ones_like(count), 1.0)
    own = m[:, 2:].astype(np.float64) - m[:, :2]
    np.testing.assert_allclose(out, own, atol=1e-12)


def test_nadaraya_watson_kernel_limits():
    # a -> 0: plain mean of the K neighbours' flows; large a with distinct
    # distances: the nearest neighbour (the match itself, distance 0) wins
    m, idx, dist, count = _random_neighbourhoods(14)
    flows = m[:, 2:].astype(np.float64) - m[:, :2]
    out0 = oracle.nw(m, idx, dist, count, 1e-12)
    np.testing.assert_allclose(out0, flows[idx].mean(axis=1), rtol=1e-9, atol=1e-9)
    far = dist.copy()
    far[:, 1:] += 0.5          # every other neighbour at least 0.5 away
    out_inf = oracle.nw(m, idx, far, count, 200.0)
    # the others' total weight is below (K-1) e^-100 relative to the match's
    np.testing.assert_allclose(out_inf, flows, atol=1e-30)
