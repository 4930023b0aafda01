"""Pins for the oracle's match graph G (Sec. 3.4, Fig. 5)."""

import numpy as np
import pytest
import scipy.sparse as sp
from scipy.sparse.csgraph import dijkstra

import oracle
from helpers import grid_graph, random_small_case, seed_pixels


def _adjacent_label_pairs(L):
    pairs = set()
    H, W = L.shape
    for dy, dx in ((0, 1), (1, 0), (1, 1), (1, -1)):
        a = L[0:H - dy, max(0, -dx):W - max(0, dx)]
        b = L[dy:H, max(0, -dx) + dx:W - max(0, dx) + dx]
        d = a != b
        for u, v in zip(a[d].ravel(), b[d].ravel()):
            pairs.add((min(u, v), max(u, v)))
    return pairs


@pytest.mark.parametrize("seed", range(5))
def test_edges_are_touching_cells(seed):
    C, m = random_small_case(100 + seed, H=22, W=26, N=12)
    D, L = oracle.geodesic(C, m)
    em, en, ew = oracle.graph(C, D, L, m)
    assert (em < en).all()
    keys = em.astype(np.int64) * m.shape[0] + en
    assert (np.diff(keys) > 0).all()          # sorted and unique
    assert set(zip(em.tolist(), en.tolist())) == _adjacent_label_pairs(L)


@pytest.mark.parametrize("seed", range(5))
def test_edge_weight_is_two_cell_restricted_geodesic(seed):
    # Sec. 3.4: the weight of (m, n) is the geodesic distance between p_m and
    # p_n with the path restricted to the union of the two cells.  Checked by
    # scipy's Dijkstra on the pixel subgraph of the two cells.
    C, m = random_small_case(200 + seed, H=20, W=20, N=9)
    H, W = C.shape
    D, L = oracle.geodesic(C, m)
    em, en, ew = oracle.graph(C, D, L, m)
    G = grid_graph(C).tocoo()
    Lf = L.ravel()
    sp_pix = seed_pixels(m, W)
    for a, b, w in zip(em, en, ew):
        keep = (Lf == a) | (Lf == b)
        sel = keep[G.row] & keep[G.col]
        sub = sp.csr_matrix((G.data[sel], (G.row[sel], G.col[sel])),
                            shape=G.shape)
        d = dijkstra(sub, directed=False, indices=[sp_pix[a]])[0, sp_pix[b]]
        assert abs(d - w) <= 1e-10 * max(d, 1.0), (a, b, d, w)


def test_graph_path_can_beat_direct_edge():
    # Fig. 5(d): the graph distance between two neighbouring matches may be
    # shorter through a third match than along their own edge.  The oracle's
    # K-NN distances must use the shortest graph path, not the direct edge.
    from paper_1501_02565_gb300 import synth
    p = synth.config_pair(1, 0)
    D, L = oracle.geodesic(p.C, p.matches)
    em, en, ew = oracle.graph(p.C, D, L, p.matches)
    G = sp.csr_matrix((np.concatenate([ew, ew]),
                       (np.concatenate([em, en]), np.concatenate([en, em]))),
                      shape=(p.N, p.N))
    Dg = dijkstra(G, directed=False)
    shorter = Dg[em, en] < ew * (1 - 1e-12)
    assert shorter.any()
    idx, dist, count = oracle.knn(p.N, em, en, ew, p.N)
    for e in np.nonzero(shorter)[0][:20]:
        a, b = em[e], en[e]
        j = int(np.nonzero(idx[a] == b)[0][0])
        assert abs(dist[a, j] - Dg[a, b]) <= 1e-12 * Dg[a, b]
        assert dist[a, j] < ew[e]


def test_duplicate_source_pixel_joins_owner_at_zero():
    C = np.ones((6, 6), np.float32)
    m = np.array([[1, 1, 0, 0], [4, 4, 0, 0], [1, 1, 0, 0]], np.float32)
    D, L = oracle.geodesic(C, m)
    em, en, ew = oracle.graph(C, D, L, m)
    e = [(a, b, w) for a, b, w in zip(em, en, ew) if (a, b) == (0, 2)]
    assert e and e[0][2] == 0.0
    idx, dist, count = oracle.knn(3, em, en, ew, 3)
    assert count[2] == 3 and idx[2, 0] == 2 and idx[2, 1] == 0
