"""The synthetic input generators (host logic, no GPU): the second frame
follows the forward flow, the smooth perturbation has the requested RMS, and
the in-frame mask is what it says."""

import numpy as np

from paper_1501_02565_gb300 import synth


def _img(H, W, seed=0):
    rng = np.random.default_rng(seed)
    ys, xs = np.mgrid[0:H, 0:W].astype(np.float64)
    img = np.zeros((H, W, 3))
    for c in range(3):
        f = rng.uniform(0.05, 0.2, 2)
        img[..., c] = 0.5 + 0.3 * np.sin(f[0] * xs + f[1] * ys + c)
    return img.astype(np.float32)


def test_second_frame_of_an_integer_translation_is_a_shift():
    I1 = _img(40, 50)
    u = np.zeros((40, 50, 2), np.float32)
    u[..., 0], u[..., 1] = 3.0, -2.0
    I2 = synth.second_frame(I1, u)
    # I2(p + u) = I1(p) wherever p + u lies inside the frame
    np.testing.assert_allclose(I2[0:38, 3:50], I1[2:40, 0:47], atol=1e-6)


def test_second_frame_follows_a_smooth_affine_forward_flow():
    # u(p) = t + B p with a small B: the fixed point v(q) = u(q - v(q)) is the
    # backward flow, so I2 sampled at p + u(p) gives back I1(p) up to the
    # bilinear interpolation of a smooth image
    H, W = 60, 80
    I1 = _img(H, W, 1)
    ys, xs = np.mgrid[0:H, 0:W].astype(np.float64)
    u = np.stack([4.0 + 0.03 * xs - 0.02 * ys, -3.0 + 0.01 * xs + 0.02 * ys], -1)
    I2 = synth.second_frame(I1, u.astype(np.float32))
    tx, ty = xs + u[..., 0], ys + u[..., 1]
    inside = (tx >= 1) & (tx <= W - 2) & (ty >= 1) & (ty <= H - 2)
    back = synth._bilinear(I2, tx, ty)
    err = np.abs(back - I1).max(-1)[inside]
    assert err.max() < 0.02, err.max()
    # the old approximation I2(q) = I1(q - u(q)) is off by |B| |u| here
    X = np.clip(xs - u[..., 0], 0, W - 1)
    Y = np.clip(ys - u[..., 1], 0, H - 1)
    old = synth._bilinear(I1, X, Y)
    err_old = np.abs(synth._bilinear(old, tx, ty) - I1).max(-1)[inside]
    assert err.mean() < 0.5 * err_old.mean()


def test_smooth_perturbation_has_the_requested_rms_and_is_smooth():
    f = synth.smooth_perturbation(120, 200, 1.5, seed=4, scale=16)
    assert f.shape == (120, 200, 2)
    assert abs(np.sqrt((f.astype(np.float64) ** 2).sum(-1).mean()) - 1.5) < 1e-4
    # bilinear between 16-px grid values: neighbouring pixels differ little
    assert np.abs(np.diff(f, axis=1)).max() < 0.5


def test_in_frame_mask():
    u = np.zeros((4, 5, 2), np.float32)
    u[..., 0] = 2.0
    m = synth.in_frame(u)
    assert m[:, :3].all() and not m[:, 3:].any()
