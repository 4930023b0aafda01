"""Pins for the image-gradient cost map (Table 2, the "||grad_2 I||_2" row)."""

import numpy as np

import oracle


def test_linear_ramp_closed_form():
    # I = alpha x + beta y: interior gradient (alpha, beta); with edge
    # replication the border differences are halved along that axis
    H, W, al, be = 9, 12, 0.03, -0.02
    ys, xs = np.mgrid[0:H, 0:W]
    C = oracle.gradient_cost(al * xs + be * ys + 0.3)
    gx = np.full((H, W), al)
    gx[:, 0] = gx[:, -1] = al / 2
    gy = np.full((H, W), be)
    gy[0, :] = gy[-1, :] = be / 2
    np.testing.assert_allclose(C, np.hypot(gx, gy), rtol=1e-12, atol=1e-15)


def test_constant_image_gives_the_floor():
    C = oracle.gradient_cost(np.full((5, 7, 3), 0.42), floor=1e-3)
    np.testing.assert_allclose(C, 1e-3, rtol=0, atol=1e-15)


def test_channels_add_in_quadrature():
    rng = np.random.default_rng(3)
    I1 = rng.uniform(0, 1, (8, 10))
    C1 = oracle.gradient_cost(I1)
    C3 = oracle.gradient_cost(np.stack([I1, I1, I1], -1))
    np.testing.assert_allclose(C3, np.sqrt(3) * C1, rtol=1e-12)


def test_transpose_symmetry_and_step_edge():
    rng = np.random.default_rng(4)
    I = rng.uniform(0, 1, (11, 6, 3))
    np.testing.assert_allclose(oracle.gradient_cost(I.transpose(1, 0, 2)),
                               oracle.gradient_cost(I).T, rtol=1e-12)
    # a vertical step of height h: the two columns beside it see h / 2
    S = np.zeros((4, 8))
    S[:, 4:] = 0.6
    C = oracle.gradient_cost(S)
    np.testing.assert_allclose(C[:, 3], 0.3, rtol=1e-12)
    np.testing.assert_allclose(C[:, 4], 0.3, rtol=1e-12)
    assert (C[:, [0, 1, 2, 5, 6, 7]] == 0).all()
