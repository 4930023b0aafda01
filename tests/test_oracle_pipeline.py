"""End-to-end pins for the oracle (Algorithm 1, LA form) and for the
approximation of Eq. 4."""

import numpy as np
import pytest

import oracle
from helpers import knn_by_scipy, load_golden, per_seed_distances, random_small_case


def test_global_affine_flow_recovered_everywhere():
    rng = np.random.default_rng(21)
    H, W, N = 40, 56, 80
    C = rng.uniform(0.01, 1.0, (H, W)).astype(np.float32)
    flat = rng.choice(H * W, N, replace=False)
    A = np.array([[0.98, 0.03], [-0.05, 1.02]])
    t = np.array([4.0, -6.0])
    m = np.zeros((N, 4), np.float32)
    m[:, 0], m[:, 1] = flat % W, flat // W
    m[:, 2:] = (m[:, :2].astype(np.float64) @ A.T + t).astype(np.float32)
    r = oracle.interp(C, m, 10, 1.0)
    ys, xs = np.mgrid[0:H, 0:W]
    P = np.stack([xs, ys], -1).astype(np.float64)
    ref = P @ A.T + t - P
    assert not r["fallback"].any()
    np.testing.assert_allclose(r["flow"], ref, atol=2e-4)


def test_piecewise_affine_recovered_away_from_walls():
    # Three regions separated by 2-px walls of high cost.  Every match's K
    # nearest graph neighbours stay in its own region, so each fit sees one
    # affine motion and is exact; pixels whose nearest match lies in their own
    # region get their region's flow.
    rng = np.random.default_rng(22)
    H, W = 48, 90
    C = np.full((H, W), 0.01, np.float32)
    C[:, 29:31] = 50.0
    C[:, 59:61] = 50.0
    region = np.zeros((H, W), np.int64)
    region[:, 30:] = 1
    region[:, 60:] = 2
    motions = [(np.array([[1.02, 0.01], [0.0, 0.99]]), np.array([3.0, 1.0])),
               (np.array([[0.97, -0.03], [0.02, 1.0]]), np.array([-8.0, 2.5])),
               (np.eye(2), np.array([12.0, -4.0]))]
    pts = []
    for r, (x0, x1) in enumerate(((0, 29), (31, 59), (61, 90))):
        cells = [(x, y) for y in range(H) for x in range(x0, x1)]
        pick = rng.choice(len(cells), 30, replace=False)
        pts += [cells[i] for i in pick]
    N = len(pts)
    m = np.zeros((N, 4), np.float32)
    for i, (x, y) in enumerate(pts):
        A, t = motions[region[y, x]]
        q = A @ np.array([x, y], float) + t
        m[i] = (x, y, q[0], q[1])
    r = oracle.interp(C, m, 12, 1.0)
    reg_of_match = region[m[:, 1].astype(int), m[:, 0].astype(int)]
    # neighbourhoods never cross a wall
    for i in range(N):
        assert (reg_of_match[r["idx"][i, :r["count"][i]]] == reg_of_match[i]).all()
    ys, xs = np.mgrid[0:H, 0:W]
    ok = reg_of_match[r["L"]] == region
    assert ok.mean() > 0.9
    for k, (A, t) in enumerate(motions):
        sel = ok & (region == k)
        P = np.stack([xs[sel], ys[sel]], -1).astype(np.float64)
        ref = P @ A.T + t - P
        np.testing.assert_allclose(r["flow"][sel], ref, atol=1e-4)


@pytest.mark.parametrize("seed", range(3))
def test_approximate_distance_upper_bounds_geodesic(seed):
    # Eq. 4: D~(p, p_n) = D_G(p, L(p)) + D^G(L(p), p_n) is the length of a real
    # path from p to p_n, so it can never be shorter than D_G(p, p_n).
    C, m = random_small_case(400 + seed, H=16, W=18, N=8)
    N = m.shape[0]
    D, L = oracle.geodesic(C, m)
    em, en, ew = oracle.graph(C, D, L, m)
    _, _, _, Dg = knn_by_scipy(N, em, en, ew, N)
    Dexact = per_seed_distances(C, m)            # [N, P]
    Lf, Df = L.ravel(), D.ravel()
    Dtilde = Df[None, :] + Dg[Lf].T              # [N, P]
    assert (Dtilde >= Dexact - 1e-9).all()
    # equality for the pixel's own match (second term is zero)
    np.testing.assert_allclose(Dtilde[Lf, np.arange(len(Lf))], Df, atol=0)


def test_approximate_distance_is_exact_along_a_chain_of_cells():
    # Eq. 4 on a one-row strip: the cells are consecutive intervals, G is the
    # chain of neighbouring matches, and each edge weight is the geodesic
    # between the two seeds.  For a pixel whose own seed lies between it and
    # p_n, the shortest path passes through that seed, so D~ equals D_G
    # exactly; for a pixel strictly between its seed and p_n it is longer.
    rng = np.random.default_rng(31)
    W = 48
    C = rng.uniform(0.05, 2.0, (1, W)).astype(np.float32)
    xs = np.array([2, 9, 17, 18, 26, 35, 44])
    N = len(xs)
    m = np.zeros((N, 4), np.float32)
    m[:, 0] = xs
    m[:, 2] = xs + 1.0
    D, L = oracle.geodesic(C, m)
    em, en, ew = oracle.graph(C, D, L, m)
    pairs = sorted(zip(np.minimum(em, en).tolist(), np.maximum(em, en).tolist()))
    assert pairs == [(i, i + 1) for i in range(N - 1)]
    _, _, _, Dg = knn_by_scipy(N, em, en, ew, N)
    Dexact = per_seed_distances(C, m)            # [N, W]
    Lf, Df = L.ravel(), D.ravel()
    Dtilde = Df[None, :] + Dg[Lf].T              # [N, W]
    seed_x = xs[Lf]                              # x of each pixel's own seed
    px = np.arange(W)
    n_eq = n_gt = 0
    for n in range(N):
        through = (seed_x - px) * (xs[n] - seed_x) >= 0
        np.testing.assert_allclose(Dtilde[n, through], Dexact[n, through], rtol=1e-12)
        n_eq += through.sum()
        beyond = ~through
        assert (Dtilde[n, beyond] > Dexact[n, beyond] + 1e-3).all()
        n_gt += beyond.sum()
    assert n_eq > 0 and n_gt > 0


def test_piecewise_property_same_knn_set_for_whole_cell():
    # Sec. 3.4 "Piecewise field": under D~, every pixel of a cell has the same
    # K nearest matches as the cell's match, and weights differ by a common
    # factor, so the per-pixel fit equals the per-match fit.  Check by fitting
    # a few pixels individually with numpy on D~.
    from helpers import lstsq_model
    C, m = random_small_case(500, H=20, W=22, N=14)
    N = m.shape[0]
    K = 6
    r = oracle.interp(C, m, K, 1.0)
    em, en, ew = r["em"], r["en"], r["ew"]
    _, _, _, Dg = knn_by_scipy(N, em, en, ew, N)
    H, W = C.shape
    rng = np.random.default_rng(1)
    for pix in rng.choice(H * W, 25, replace=False):
        y, x = divmod(int(pix), W)
        l = r["L"][y, x]
        dt = r["D"][y, x] + Dg[l]
        order = np.lexsort((np.arange(N), dt))[:K]
        assert set(order) == set(r["idx"][l, :r["count"][l]])
        ref = lstsq_model(m, l, order, dt[order], 1.0)
        flow = ref[:2] + np.array([[ref[2], ref[3]], [ref[4], ref[5]]]) @ (
            np.array([x, y], float) - m[l, :2])
        np.testing.assert_allclose(r["flow"][y, x], flow, rtol=1e-7, atol=1e-7)


@pytest.mark.parametrize("K", [3, 2])
def test_hand_derived_strip_through_every_stage(K):
    # tests/golden/pipeline_strip.txt: labels, distances, graph, K-NN lists
    # (with an index tie), the NW fallback of a degenerate fit and the
    # dense flow, all worked out by hand
    g = load_golden("pipeline_strip.txt")
    a = float(g["a"][0])
    r = oracle.interp(g["C"], g["matches"], K, a)
    np.testing.assert_allclose(r["D"], g["D"], rtol=0, atol=1e-12)
    np.testing.assert_array_equal(r["L"], g["L"])
    edges = sorted(zip(np.minimum(r["em"], r["en"]), np.maximum(r["em"], r["en"]), r["ew"]))
    np.testing.assert_allclose(np.array(edges, float).ravel(), g["edges"], rtol=0, atol=1e-12)
    np.testing.assert_array_equal(r["idx"][:, :K].ravel(), g[f"K{K}_idx"])
    np.testing.assert_allclose(r["dist"][:, :K].ravel(), g[f"K{K}_dist"], rtol=0, atol=1e-12)
    assert r["fallback"].all()
    per_match = np.stack([g[f"K{K}_flow_u"], g[f"K{K}_flow_v"]], -1)
    np.testing.assert_allclose(r["flow"][0], per_match[g["L"][0]], rtol=0, atol=1e-12)


@pytest.mark.parametrize("a", [0.05, 0.5, 1.0])
def test_hand_derived_affine_triangle(a):
    # tests/golden/affine_triangle.txt: three correspondences fix one affine
    # map, which the LA fit must return for every match and every pixel
    g = load_golden("affine_triangle.txt")
    r = oracle.interp(g["C"], g["matches"], 3, a)
    assert not r["fallback"].any()
    model = r["model"]                           # (c_u, c_v, b11, b12, b21, b22)
    np.testing.assert_allclose(model[:, :2].ravel(), g["c"], rtol=0, atol=1e-12)
    np.testing.assert_allclose(model[:, 2:], np.tile(g["B"], (3, 1)), rtol=0, atol=1e-12)
    np.testing.assert_allclose(r["flow"][..., 0], np.repeat(g["flow_u_by_row"][:, None], 5, 1),
                               rtol=0, atol=1e-12)
    np.testing.assert_allclose(r["flow"][..., 1], np.repeat(g["flow_v_by_col"][None, :], 5, 0),
                               rtol=0, atol=1e-12)
