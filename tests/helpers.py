"""Independent checkers used to pin the oracle and to compare the CUDA path.

Nothing here calls the oracle's C code: the pixel graph is built with numpy
and solved with scipy's Dijkstra, least squares goes through numpy's SVD
solver, and fixtures are parsed from hand-derived text files.
"""

from __future__ import annotations

import os

import numpy as np
import scipy.sparse as sp
from scipy.sparse.csgraph import dijkstra

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def load_golden(name):
    """Parse a `key v1 v2 ...` fixture, ignoring # comments."""
    out = {}
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.split("#", 1)[0].strip()
            if not line:
                continue
            k, *vals = line.split()
            out[k] = np.array([float(v) for v in vals])
    H, W = int(out["H"][0]), int(out["W"][0])
    out["H"], out["W"] = H, W
    out["C"] = out["C"].reshape(H, W).astype(np.float32)
    out["matches"] = out["matches"].reshape(-1, 4).astype(np.float32)
    if "D" in out:
        out["D"] = out["D"].reshape(H, W)
    if "L" in out:
        out["L"] = out["L"].reshape(H, W).astype(np.int64)
    return out


def grid_graph(C):
    """scipy CSR of the 8-connected pixel grid; the step p-q costs
    |p-q| (C(p)+C(q))/2 (Eq. 3 discretised by the trapezoid rule)."""
    H, W = C.shape
    Cd = C.astype(np.float64)
    idx = np.arange(H * W).reshape(H, W)
    rows, cols, vals = [], [], []
    for dy, dx in ((0, 1), (1, 0), (1, 1), (1, -1)):
        y0, y1 = 0, H - dy
        x0, x1 = max(0, -dx), W - max(0, dx)
        a = idx[y0:y1, x0:x1]
        b = idx[y0 + dy:y1 + dy, x0 + dx:x1 + dx]
        ln = np.sqrt(2.0) if (dx and dy) else 1.0
        w = ln * (Cd[y0:y1, x0:x1] + Cd[y0 + dy:y1 + dy, x0 + dx:x1 + dx]) / 2
        rows += [a.ravel(), b.ravel()]
        cols += [b.ravel(), a.ravel()]
        vals += [w.ravel(), w.ravel()]
    r = np.concatenate(rows)
    c = np.concatenate(cols)
    v = np.concatenate(vals)
    # zero-cost steps would be dropped by the sparse format; keep them with
    # a tiny positive placeholder is wrong, so callers use C > 0.
    return sp.csr_matrix((v, (r, c)), shape=(H * W, H * W))


def seed_pixels(matches, W):
    x = np.floor(matches[:, 0].astype(np.float64) + 0.5).astype(np.int64)
    y = np.floor(matches[:, 1].astype(np.float64) + 0.5).astype(np.int64)
    return y * W + x


def per_seed_distances(C, matches):
    """[N, P] geodesic distance from every match to every pixel."""
    G = grid_graph(C)
    return dijkstra(G, directed=False, indices=seed_pixels(matches, C.shape[1]))


def brute_assignment(C, matches):
    """D = min over matches, L = smallest index among the minimisers, and a
    mask of pixels whose best two matches are within 1e-12 relative."""
    Dm = per_seed_distances(C, matches)
    L = np.argmin(Dm, axis=0)  # argmin returns the first (smallest) index
    D = Dm[L, np.arange(Dm.shape[1])]
    srt = np.sort(Dm, axis=0)
    if Dm.shape[0] > 1:
        tie = (srt[1] - srt[0]) <= 1e-12 * np.maximum(srt[0], 1e-300)
    else:
        tie = np.zeros(Dm.shape[1], bool)
    H, W = C.shape
    return D.reshape(H, W), L.reshape(H, W), tie.reshape(H, W), Dm


def match_graph_csr(N, em, en, ew):
    return sp.csr_matrix(
        (np.concatenate([ew, ew]),
         (np.concatenate([em, en]), np.concatenate([en, em]))),
        shape=(N, N))


def knn_by_scipy(N, em, en, ew, K):
    """K nearest matches of every match on G under (distance, index) order."""
    G = match_graph_csr(N, em, en, ew)
    Dg = dijkstra(G, directed=False)
    idx = np.full((N, K), -1, np.int64)
    dist = np.full((N, K), np.inf)
    near_tie = np.zeros(N, bool)
    for m in range(N):
        d = Dg[m]
        order = np.lexsort((np.arange(N), d))
        order = order[np.isfinite(d[order])]
        k = min(K, len(order))
        idx[m, :k] = order[:k]
        dist[m, :k] = d[order[:k]]
        if len(order) > K:
            dk, dk1 = d[order[K - 1]], d[order[K]]
            near_tie[m] = (dk1 - dk) <= 1e-9 * max(dk, 1e-300)
    return idx, dist, near_tie, Dg


def lstsq_model(matches, m, nbrs, d, a, weight_squared=True):
    """Independent LA fit at match m: rows [x~, y~, 1] -> (u, v), each row
    scaled by sqrt(weight) and solved by numpy's SVD least squares."""
    mt = matches.astype(np.float64)
    xm, ym = mt[m, 0], mt[m, 1]
    k = np.exp(-a * np.asarray(d, np.float64))
    w = k * k if weight_squared else k
    s = np.sqrt(w)
    X = np.stack([mt[nbrs, 0] - xm, mt[nbrs, 1] - ym, np.ones(len(nbrs))], 1)
    U = mt[nbrs, 2] - mt[nbrs, 0]
    V = mt[nbrs, 3] - mt[nbrs, 1]
    bu = np.linalg.lstsq(X * s[:, None], U * s, rcond=None)[0]
    bv = np.linalg.lstsq(X * s[:, None], V * s, rcond=None)[0]
    return np.array([bu[2], bv[2], bu[0], bu[1], bv[0], bv[1]])


def random_small_case(seed, H=20, W=24, N=10, c_lo=0.05, c_hi=2.0):
    """Random positive cost map and N distinct match pixels (tiny inputs)."""
    rng = np.random.default_rng(seed)
    C = rng.uniform(c_lo, c_hi, size=(H, W)).astype(np.float32)
    flat = rng.choice(H * W, N, replace=False)
    m = np.zeros((N, 4), np.float32)
    m[:, 0] = flat % W
    m[:, 1] = flat // W
    m[:, 2] = m[:, 0] + rng.normal(0, 3, N)
    m[:, 3] = m[:, 1] + rng.normal(0, 3, N)
    return C, m
