"""FP64 oracle of the variational refinement (Sec. 4, "Variational Energy
Minimization").  TEST INFRASTRUCTURE ONLY, like the rest of this package.

The paper fixes the structure and leaves the constants to its references:
the energy is a data term (colour constancy and gradient constancy with a
normalisation factor, after Zimmer et al.) plus a smoothness term on the
flow gradient with the local weight alpha(x) = exp(-kappa ||grad I(x)||),
kappa = 5; it is minimised from the interpolated flow at full resolution by
5 fixed-point iterations (re-linearise, recompute the non-linear weights,
solve for the update) with 30 SOR iterations per linear system.  The
readings taken here (each listed in the design notes):

  * images in [0, 1]; derivatives are central differences on the
    edge-replicated image (the cost-map operator);
  * one iteration: warp I2 by the current flow (bilinear, coordinates
    clamped to the image), linearise at the current flow, take the
    non-linear weights at zero update (lagged), solve for the update (du, dv)
    from zero, add it to the flow;
  * derivatives of the linearised constancies average the two frames:
    I_x = (D_x I1 + D_x I2w) / 2 and so on, I_z = I2w - I1; gradient
    constancy uses the gradient images G_x = D_x I, G_y = D_y I in the same
    way;
  * normalisation theta = 1 / (|grad|^2 + zeta^2) per channel and term;
  * robust penaliser Psi(s^2) = sqrt(s^2 + eps^2), applied once to the
    colour term and once to the gradient term (summed over channels);
  * smoothness weight phi = alpha(x) Psi'(|grad u|^2 + |grad v|^2) per
    pixel, alpha = alpha0 exp(-kappa ||grad I1||); the weight of the edge
    between 4-neighbours p, q is (phi(p) + phi(q)) / 2; no flux across the
    image border;
  * SOR in red-black order (red: x + y even), red then black in every
    iteration; at each pixel the 2 x 2 system coupling du and dv is solved
    exactly (point-coupled SOR) and both are over-relaxed by omega.
"""

from __future__ import annotations

import dataclasses

import numpy as np


@dataclasses.dataclass(frozen=True)
class RefineParams:
    alpha0: float = 1.0     # smoothness weight scale
    gamma: float = 0.7      # weight of the gradient constancy term
    kappa: float = 5.0      # edge sensitivity of alpha (Sec. 4)
    eps: float = 1e-3       # robust penaliser
    zeta: float = 0.1       # normalisation
    omega: float = 1.6      # SOR relaxation
    iterations: int = 5     # fixed-point iterations (Sec. 4)
    sor_iterations: int = 30  # SOR iterations per linear system (Sec. 4)


def _pad(a):
    return np.pad(a, ((1, 1), (1, 1)) + ((0, 0),) * (a.ndim - 2), mode="edge")


def dx(a):
    p = _pad(a)
    return (p[1:-1, 2:] - p[1:-1, :-2]) / 2.0


def dy(a):
    p = _pad(a)
    return (p[2:, 1:-1] - p[:-2, 1:-1]) / 2.0


def warp_bilinear(I, u, v):
    """I [H, W, C] sampled at (x + u, y + v), coordinates clamped to the
    image, bilinear."""
    H, W = I.shape[:2]
    ys, xs = np.mgrid[0:H, 0:W].astype(np.float64)
    X = np.clip(xs + u, 0.0, W - 1.0)
    Y = np.clip(ys + v, 0.0, H - 1.0)
    x0 = np.minimum(np.floor(X).astype(np.int64), W - 2) if W > 1 else np.zeros_like(X, np.int64)
    y0 = np.minimum(np.floor(Y).astype(np.int64), H - 2) if H > 1 else np.zeros_like(Y, np.int64)
    x1 = np.minimum(x0 + 1, W - 1)
    y1 = np.minimum(y0 + 1, H - 1)
    ax = (X - x0)[..., None]
    ay = (Y - y0)[..., None]
    return ((1 - ay) * ((1 - ax) * I[y0, x0] + ax * I[y0, x1]) +
            ay * ((1 - ax) * I[y1, x0] + ax * I[y1, x1]))


def coefficients(I1, I2w, u, v, prm: RefineParams):
    """Per-pixel linear system of one fixed-point iteration:
    A11, A12, A22, b1, b2 (data term, lagged weights) and phi (smoothness)."""
    z2 = prm.zeta ** 2

    def dpsi(s2):
        return 0.5 / np.sqrt(s2 + prm.eps ** 2)

    # colour constancy
    Ix = 0.5 * (dx(I1) + dx(I2w))
    Iy = 0.5 * (dy(I1) + dy(I2w))
    Iz = I2w - I1
    t0 = 1.0 / (Ix * Ix + Iy * Iy + z2)
    # gradient constancy on G_x = D_x I and G_y = D_y I
    G1x, G1y, G2x, G2y = dx(I1), dy(I1), dx(I2w), dy(I2w)
    Ixx = 0.5 * (dx(G1x) + dx(G2x))
    Ixy = 0.5 * (dy(G1x) + dy(G2x))
    Ixz = G2x - G1x
    Iyx = 0.5 * (dx(G1y) + dx(G2y))
    Iyy = 0.5 * (dy(G1y) + dy(G2y))
    Iyz = G2y - G1y
    tx = 1.0 / (Ixx * Ixx + Ixy * Ixy + z2)
    ty = 1.0 / (Iyx * Iyx + Iyy * Iyy + z2)
    pc = dpsi((t0 * Iz * Iz).sum(-1))
    pg = dpsi((tx * Ixz * Ixz + ty * Iyz * Iyz).sum(-1))
    g = prm.gamma
    A11 = pc * (t0 * Ix * Ix).sum(-1) + g * pg * (tx * Ixx * Ixx + ty * Iyx * Iyx).sum(-1)
    A12 = pc * (t0 * Ix * Iy).sum(-1) + g * pg * (tx * Ixx * Ixy + ty * Iyx * Iyy).sum(-1)
    A22 = pc * (t0 * Iy * Iy).sum(-1) + g * pg * (tx * Ixy * Ixy + ty * Iyy * Iyy).sum(-1)
    b1 = pc * (t0 * Ix * Iz).sum(-1) + g * pg * (tx * Ixx * Ixz + ty * Iyx * Iyz).sum(-1)
    b2 = pc * (t0 * Iy * Iz).sum(-1) + g * pg * (tx * Ixy * Ixz + ty * Iyy * Iyz).sum(-1)
    # smoothness
    grad1 = np.sqrt((dx(I1) ** 2 + dy(I1) ** 2).sum(-1))
    alpha = prm.alpha0 * np.exp(-prm.kappa * grad1)
    phi = alpha * dpsi(dx(u) ** 2 + dy(u) ** 2 + dx(v) ** 2 + dy(v) ** 2)
    return A11, A12, A22, b1, b2, phi


def sor(u, v, A11, A12, A22, b1, b2, phi, omega, iterations):
    """Red-black SOR for the update (du, dv) of one fixed-point iteration."""
    H, W = u.shape
    # edge weights: sx between (x, y) and (x + 1, y), sy between (x, y) and (x, y + 1)
    sx = np.zeros((H, W))
    sy = np.zeros((H, W))
    sx[:, :-1] = 0.5 * (phi[:, :-1] + phi[:, 1:])
    sy[:-1, :] = 0.5 * (phi[:-1, :] + phi[1:, :])
    sl = np.zeros((H, W)); sl[:, 1:] = sx[:, :-1]     # edge to the left neighbour
    su = np.zeros((H, W)); su[1:, :] = sy[:-1, :]     # edge to the upper neighbour
    S = sx + sl + sy + su
    du = np.zeros((H, W))
    dv = np.zeros((H, W))
    ys, xs = np.mgrid[0:H, 0:W]
    red = (xs + ys) % 2 == 0

    def nsum(f):
        """sum over the 4-neighbours q of s_pq * f(q) (zero weight off the image)."""
        out = np.zeros((H, W))
        out[:, :-1] += sx[:, :-1] * f[:, 1:]
        out[:, 1:] += sl[:, 1:] * f[:, :-1]
        out[:-1, :] += sy[:-1, :] * f[1:, :]
        out[1:, :] += su[1:, :] * f[:-1, :]
        return out

    a = A11 + S
    d = A22 + S
    det = a * d - A12 * A12          # > 0: A is a sum of outer products, S > 0
    ok = det > 0
    det = np.where(ok, det, 1.0)
    for _ in range(iterations):
        for colour in (red, ~red):
            r1 = nsum(u + du) - S * u - b1
            r2 = nsum(v + dv) - S * v - b2
            nu = (d * r1 - A12 * r2) / det
            nv = (a * r2 - A12 * r1) / det
            upd = colour & ok
            du = np.where(upd, (1 - omega) * du + omega * nu, du)
            dv = np.where(upd, (1 - omega) * dv + omega * nv, dv)
    return du, dv


def refine(I1, I2, flow, prm: RefineParams = RefineParams()):
    """Variational refinement of `flow` [H, W, 2] between images I1, I2
    [H, W, C] (or [H, W]); returns the refined flow, float64."""
    I1 = np.asarray(I1, np.float64)
    I2 = np.asarray(I2, np.float64)
    if I1.ndim == 2:
        I1, I2 = I1[..., None], I2[..., None]
    u = np.array(flow[..., 0], np.float64)
    v = np.array(flow[..., 1], np.float64)
    for _ in range(prm.iterations):
        I2w = warp_bilinear(I2, u, v)
        A11, A12, A22, b1, b2, phi = coefficients(I1, I2w, u, v, prm)
        du, dv = sor(u, v, A11, A12, A22, b1, b2, phi, prm.omega, prm.sor_iterations)
        u = u + du
        v = v + dv
    return np.stack([u, v], -1)
