"""Pins for the variational refinement oracle (Sec. 4, "Variational Energy
Minimization": data term with colour and gradient constancy, smoothness
weighted by exp(-kappa ||grad I||), 5 fixed-point x 30 SOR iterations)."""

import numpy as np
import scipy.sparse as sp
from scipy.sparse.linalg import spsolve

from oracle import refine as R


def _texture(H, W, seed, C=3):
    rng = np.random.default_rng(seed)
    ys, xs = np.mgrid[0:H, 0:W].astype(np.float64)
    img = np.zeros((H, W, C))
    for c in range(C):
        for _ in range(3):
            f = rng.uniform(0.1, 0.5, 2)
            img[..., c] += rng.uniform(0.05, 0.15) * np.sin(f[0] * xs + f[1] * ys + rng.uniform(0, 6))
    return 0.5 + img


def test_bilinear_warp_is_exact_on_a_ramp():
    H, W = 7, 9
    ys, xs = np.mgrid[0:H, 0:W].astype(np.float64)
    I = (0.03 * xs - 0.02 * ys + 0.4)[..., None]
    rng = np.random.default_rng(1)
    u = rng.uniform(-1.5, 1.5, (H, W))
    v = rng.uniform(-1.5, 1.5, (H, W))
    X = np.clip(xs + u, 0, W - 1)
    Y = np.clip(ys + v, 0, H - 1)
    np.testing.assert_allclose(R.warp_bilinear(I, u, v)[..., 0], 0.03 * X - 0.02 * Y + 0.4,
                               rtol=0, atol=1e-14)


def test_identical_frames_and_zero_flow_stay_put():
    I = _texture(12, 15, 2)
    out = R.refine(I, I, np.zeros((12, 15, 2)))
    assert np.abs(out).max() < 1e-12


def test_sor_converges_to_the_direct_solution():
    # many SOR iterations solve the assembled linear system: compare with a
    # sparse direct solve of the same equations, built independently
    H, W = 9, 11
    I1 = _texture(H, W, 3)
    I2 = _texture(H, W, 4)
    rng = np.random.default_rng(5)
    u = rng.normal(0, 0.5, (H, W))
    v = rng.normal(0, 0.5, (H, W))
    prm = R.RefineParams()
    A11, A12, A22, b1, b2, phi = R.coefficients(I1, R.warp_bilinear(I2, u, v), u, v, prm)
    du, dv = R.sor(u, v, A11, A12, A22, b1, b2, phi, 1.6, 3000)
    n = H * W
    idx = np.arange(n).reshape(H, W)
    rows, cols, vals = [], [], []
    rhs = np.zeros(2 * n)
    for y in range(H):
        for x in range(W):
            p = idx[y, x]
            rows += [p, p, n + p, n + p]
            cols += [p, n + p, p, n + p]
            vals += [A11[y, x], A12[y, x], A12[y, x], A22[y, x]]
            rhs[p] -= b1[y, x]
            rhs[n + p] -= b2[y, x]
            for qy, qx in ((y, x + 1), (y, x - 1), (y + 1, x), (y - 1, x)):
                if 0 <= qx < W and 0 <= qy < H:
                    s = 0.5 * (phi[y, x] + phi[qy, qx])
                    q = idx[qy, qx]
                    for off, f in ((0, u), (n, v)):
                        rows += [off + p, off + p]
                        cols += [off + p, off + q]
                        vals += [s, -s]
                        rhs[off + p] += s * (f[qy, qx] - f[y, x])
    M = sp.csr_matrix((vals, (rows, cols)), shape=(2 * n, 2 * n))
    ref = spsolve(M, rhs)
    np.testing.assert_allclose(du.ravel(), ref[:n], rtol=1e-8, atol=1e-10)
    np.testing.assert_allclose(dv.ravel(), ref[n:], rtol=1e-8, atol=1e-10)


def test_transpose_symmetry():
    H, W = 10, 13
    I1 = _texture(H, W, 6)
    I2 = _texture(H, W, 7)
    f = np.random.default_rng(8).normal(0, 0.7, (H, W, 2))
    a = R.refine(I1, I2, f)
    b = R.refine(I1.transpose(1, 0, 2), I2.transpose(1, 0, 2), f.transpose(1, 0, 2)[..., ::-1])
    np.testing.assert_allclose(b.transpose(1, 0, 2)[..., ::-1], a, rtol=1e-9, atol=1e-11)


def test_refinement_recovers_a_translation():
    # I2 is I1 moved by (2, 1) (sampled from the same analytic texture); a
    # flow off by up to half a pixel is pulled back to the translation
    H, W = 40, 48
    rng = np.random.default_rng(9)
    ys, xs = np.mgrid[0:H, 0:W].astype(np.float64)
    waves = [(rng.uniform(0.15, 0.45, 2), rng.uniform(0, 6), rng.uniform(0.05, 0.12))
             for _ in range(6)]

    def tex(X, Y):
        out = np.zeros((H, W, 3)) + 0.5
        for c in range(3):
            for k, (fq, ph, am) in enumerate(waves):
                out[..., c] += am * np.sin(fq[0] * X + fq[1] * Y + ph + c * k)
        return out

    I1 = tex(xs, ys)
    I2 = tex(xs - 2.0, ys - 1.0)
    f0 = np.stack([2.0 + rng.uniform(-0.5, 0.5, (H, W)), 1.0 + rng.uniform(-0.5, 0.5, (H, W))], -1)
    out = R.refine(I1, I2, f0)
    inner = (slice(4, -4), slice(4, -4))
    e0 = np.hypot(f0[..., 0] - 2, f0[..., 1] - 1)[inner].mean()
    e1 = np.hypot(out[..., 0] - 2, out[..., 1] - 1)[inner].mean()
    assert e1 < 0.2 * e0, (e0, e1)


def _load_fixture(name):
    import os
    out = {}
    with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", name)) as f:
        for line in f:
            line = line.split("#", 1)[0].strip()
            if line:
                k, *vals = line.split()
                out[k] = [float(v) for v in vals]
    return out


def test_coefficients_match_the_hand_derived_fixture():
    # tests/golden/refine_coeffs.txt: two-channel quadratic frames on 7x7,
    # where central differences are exact, with every term of the data and
    # smoothness coefficients derived by hand at two pixels.  Dropping the
    # normalisation theta or gamma, weighting by exp(-kappa ||grad I||^2),
    # sharing one Psi between the two constancies, or taking Psi' at another
    # residual changes these values.
    g = _load_fixture("refine_coeffs.txt")
    ys, xs = np.mgrid[0:7, 0:7].astype(np.float64)
    X, Y = xs - 3, ys - 3
    I1 = np.stack([0.5 + 0.4 * X + 0.2 * Y + 0.1 * X * X + 0.05 * X * Y - 0.05 * Y * Y,
                   0.3 - 0.2 * X + 0.1 * Y + 0.1 * X * Y], -1)
    I2w = I1 + np.stack([0.1 + 0.02 * X - 0.04 * Y + 0.1 * Y * Y,
                         -0.05 + 0.06 * X + 0.02 * X * X], -1)
    u = 0.2 * X + 0.1 * Y
    v = -0.1 * X + 0.3 * Y
    out = dict(zip(("A11", "A12", "A22", "b1", "b2", "phi"),
                   R.coefficients(I1, I2w, u, v, R.RefineParams())))
    for tag in ("3_3", "4_2"):
        x, y = (int(t) for t in g["at_" + tag])
        for k, arr in out.items():
            np.testing.assert_allclose(arr[y, x], g[f"{k}_{tag}"][0], rtol=1e-12, atol=1e-15,
                                       err_msg=f"{k} at ({x},{y})")
