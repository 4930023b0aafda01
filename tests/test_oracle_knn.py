"""Pins for N_K(p_m) by Dijkstra on G (Algorithm 1 step 5, Sec. 3.2)."""

import numpy as np
import pytest

import oracle
from helpers import knn_by_scipy, random_small_case


def _check(N, em, en, ew, K):
    idx, dist, count = oracle.knn(N, em, en, ew, K)
    ridx, rdist, near_tie, Dg = knn_by_scipy(N, em, en, ew, K)
    for m in range(N):
        reach = int(np.isfinite(Dg[m]).sum())
        assert count[m] == min(K, reach)
        c = count[m]
        assert idx[m, 0] == m and dist[m, 0] == 0.0   # p_m is its own nearest
        np.testing.assert_allclose(dist[m, :c], rdist[m, :c], rtol=1e-12,
                                   atol=0)
        if not near_tie[m]:
            assert (idx[m, :c] == ridx[m, :c]).all()
        else:
            assert set(idx[m, :c - 1]) <= set(ridx[m, :c]) | set(idx[m, :c])
    return idx, dist, count


@pytest.mark.parametrize("seed", range(4))
def test_knn_matches_scipy_on_pixel_graphs(seed):
    C, m = random_small_case(300 + seed, H=30, W=34, N=40)
    D, L = oracle.geodesic(C, m)
    em, en, ew = oracle.graph(C, D, L, m)
    for K in (1, 3, 10, 40):
        _check(40, em, en, ew, K)


def test_knn_on_random_graph_with_components_and_ties():
    rng = np.random.default_rng(7)
    N = 60
    # two components; integer weights make exact distance ties common
    em, en = [], []
    for comp in (range(0, 35), range(35, 60)):
        comp = list(comp)
        for i in range(1, len(comp)):
            em.append(comp[rng.integers(0, i)])
            en.append(comp[i])
        for _ in range(len(comp)):
            a, b = rng.choice(comp, 2, replace=False)
            em.append(a)
            en.append(b)
    pairs = {(min(a, b), max(a, b)) for a, b in zip(em, en)}
    em = np.array([p[0] for p in sorted(pairs)], np.int32)
    en = np.array([p[1] for p in sorted(pairs)], np.int32)
    ew = rng.integers(1, 4, size=len(em)).astype(np.float64)
    idx, dist, count = _check(N, em, en, ew, 30)
    assert count[0] == 30 and count[40] == 25
    # ties at equal distance are settled in increasing index order
    for m in range(N):
        c = count[m]
        for j in range(1, c):
            assert (dist[m, j - 1], idx[m, j - 1]) < (dist[m, j], idx[m, j])


def test_single_match_graph():
    idx, dist, count = oracle.knn(1, np.zeros(0, np.int32),
                                  np.zeros(0, np.int32), np.zeros(0), 5)
    assert count[0] == 1 and idx[0, 0] == 0 and dist[0, 0] == 0
