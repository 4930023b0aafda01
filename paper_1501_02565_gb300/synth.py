"""Seeded synthetic workloads for the sparse-to-dense interpolator.

This module produces inputs only: an edge-cost map C, a sparse match set
M = {(p_m, p'_m)} and the ground-truth dense flow the matches were drawn from.
It holds none of the interpolation arithmetic, so the CPU oracle and the CUDA
path can both consume its output without sharing any of the method.

The shapes follow the workloads the paper evaluates on (Sec. 3.1: about 5000
matches for a 1024x436 frame, one match per ~90 pixels; Sec. 3.3: C is an
image-edge map standing in for motion boundaries; Sec. 5: K ~ 100 and a ~ 1
for the LA estimator).  No dataset item is reproduced: regions, motions and
matches are random draws from a numpy PCG64 generator seeded with
``1000 * config + pair_index``.

Layout conventions (shared with the C ABI):
  * C      float32 [H, W], row-major, finite, >= 1e-3.
  * matches float32 [N, 4] rows (x, y, x', y'), x = column, y = row; the
    source position (x, y) is an integral pixel centre inside the image and
    no two matches share a source pixel.
  * gt_flow float32 [H, W, 2] (u, v) = p' - p.
"""

from __future__ import annotations

import dataclasses
import math

import numpy as np

__all__ = [
    "Pair",
    "make_polygon_pair",
    "make_kitti_pair",
    "config_pair",
    "batch_pairs",
    "serving_requests",
    "CONFIG_NAMES",
]

CONFIG_NAMES = {
    1: "single pair 256x128, 6 polygon regions, N=500, K=32",
    2: "Sintel-shaped pair 1024x436, 40 regions, N=5000, K=100",
    3: "KITTI-shaped pair 1242x375, ground plane + 20 boxes, N=8000, K=100",
    4: "batch of 64 mixed-size pairs, N=P/100, K in {64,100,128}",
    5: "serving stream, Poisson arrivals, mixed sizes, N<=30000, K=100",
}


@dataclasses.dataclass
class Pair:
    """One frame pair's interpolation inputs plus the flow they came from."""

    H: int
    W: int
    C: np.ndarray          # float32 [H, W]
    matches: np.ndarray    # float32 [N, 4]
    gt_flow: np.ndarray    # float32 [H, W, 2]
    K: int
    a: float
    name: str = ""
    regions: np.ndarray | None = None   # int32 [H, W] region map (for images)

    @property
    def N(self) -> int:
        return int(self.matches.shape[0])

    @property
    def P(self) -> int:
        return self.H * self.W


# ----------------------------------------------------------------------------
# geometry helpers (pure input construction)
# ----------------------------------------------------------------------------

def _hull(pts: np.ndarray) -> np.ndarray:
    """Counter-clockwise convex hull (monotone chain) of a few 2-D points."""
    pts = np.unique(np.round(pts, 6), axis=0)
    pts = pts[np.lexsort((pts[:, 1], pts[:, 0]))]
    if len(pts) < 3:
        return pts

    def cross(o, a, b):
        return (a[0] - o[0]) * (b[1] - o[1]) - (a[1] - o[1]) * (b[0] - o[0])

    lower, upper = [], []
    for p in pts:
        while len(lower) >= 2 and cross(lower[-2], lower[-1], p) <= 0:
            lower.pop()
        lower.append(p)
    for p in pts[::-1]:
        while len(upper) >= 2 and cross(upper[-2], upper[-1], p) <= 0:
            upper.pop()
        upper.append(p)
    return np.array(lower[:-1] + upper[:-1])


def _paint_convex(R: np.ndarray, poly: np.ndarray, rid: int) -> None:
    """Set R to rid at every pixel centre inside the convex polygon."""
    H, W = R.shape
    if len(poly) < 3:
        return
    x0 = max(int(math.floor(poly[:, 0].min())), 0)
    x1 = min(int(math.ceil(poly[:, 0].max())), W - 1)
    y0 = max(int(math.floor(poly[:, 1].min())), 0)
    y1 = min(int(math.ceil(poly[:, 1].max())), H - 1)
    if x1 < x0 or y1 < y0:
        return
    ys, xs = np.mgrid[y0:y1 + 1, x0:x1 + 1]
    inside = np.ones(xs.shape, dtype=bool)
    n = len(poly)
    for i in range(n):
        ax, ay = poly[i]
        bx, by = poly[(i + 1) % n]
        inside &= (bx - ax) * (ys - ay) - (by - ay) * (xs - ax) >= 0
    R[y0:y1 + 1, x0:x1 + 1][inside] = rid


def _boundary_strength(R: np.ndarray, strength: np.ndarray) -> np.ndarray:
    """Edge magnitude: at p, the max region strength over 4-neighbours q with
    R(q) != R(p).  Both sides of a boundary are marked, so every boundary is
    at least two pixels wide and 4-connected (no diagonal gaps)."""
    E = np.zeros(R.shape, dtype=np.float32)
    S = strength[R]
    for dy, dx in ((0, 1), (1, 0)):
        a = R[: R.shape[0] - dy, : R.shape[1] - dx]
        b = R[dy:, dx:]
        diff = a != b
        s = np.maximum(S[: R.shape[0] - dy, : R.shape[1] - dx], S[dy:, dx:])
        s = np.where(diff, s, 0.0).astype(np.float32)
        Ea = E[: R.shape[0] - dy, : R.shape[1] - dx]
        Eb = E[dy:, dx:]
        np.maximum(Ea, s, out=Ea)
        np.maximum(Eb, s, out=Eb)
    return E


def _affine_flow(R: np.ndarray, motions: list) -> np.ndarray:
    """Dense ground-truth flow: pixel p in region r moves to
    c_r + A_r (p - c_r) + t_r."""
    H, W = R.shape
    ys, xs = np.mgrid[0:H, 0:W].astype(np.float64)
    flow = np.zeros((H, W, 2), dtype=np.float64)
    for rid, (c, A, t) in enumerate(motions):
        m = R == rid
        if not m.any():
            continue
        dx = xs[m] - c[0]
        dy = ys[m] - c[1]
        nx = c[0] + A[0, 0] * dx + A[0, 1] * dy + t[0]
        ny = c[1] + A[1, 0] * dx + A[1, 1] * dy + t[1]
        flow[m, 0] = nx - xs[m]
        flow[m, 1] = ny - ys[m]
    return flow


def _region_motion(rng, R, rid, t_range, lin_range):
    ys, xs = np.nonzero(R == rid)
    if len(xs):
        c = np.array([xs.mean(), ys.mean()])
    else:
        c = np.array([0.0, 0.0])
    A = np.eye(2) + rng.uniform(-lin_range, lin_range, size=(2, 2))
    t = rng.uniform(-t_range, t_range, size=2)
    return (c, A, t)


def _cost_from_edges(rng, E: np.ndarray, sigma: float) -> np.ndarray:
    noisy = E.astype(np.float64) + rng.normal(0.0, sigma, size=E.shape)
    return (1e-3 + np.maximum(noisy, 0.0)).astype(np.float32)


def _make_matches(rng, gt_flow, xs, ys, noise_sd, outlier_frac, R_out):
    n = len(xs)
    u = gt_flow[ys, xs, 0] + rng.normal(0.0, noise_sd, size=n)
    v = gt_flow[ys, xs, 1] + rng.normal(0.0, noise_sd, size=n)
    n_out = int(round(outlier_frac * n))
    if n_out:
        idx = rng.choice(n, n_out, replace=False)
        u[idx] = rng.uniform(-R_out, R_out, size=n_out)
        v[idx] = rng.uniform(-R_out, R_out, size=n_out)
    m = np.empty((n, 4), dtype=np.float32)
    m[:, 0] = xs
    m[:, 1] = ys
    m[:, 2] = (xs + u).astype(np.float32)
    m[:, 3] = (ys + v).astype(np.float32)
    return m


def _jittered_grid(rng, H, W, N, spacing=8, jitter=3):
    """Exactly N distinct pixels drawn without replacement from a jittered
    grid of the given spacing (falls back to uniform pixels if the grid is
    too coarse for N)."""
    gx = np.arange(spacing // 2, W, spacing)
    gy = np.arange(spacing // 2, H, spacing)
    if len(gx) * len(gy) < N:
        flat = rng.choice(H * W, N, replace=False)
        return (flat % W).astype(np.int64), (flat // W).astype(np.int64)
    GX, GY = np.meshgrid(gx, gy)
    GX = GX.ravel()
    GY = GY.ravel()
    pick = rng.choice(len(GX), N, replace=False)
    xs = np.clip(GX[pick] + rng.integers(-jitter, jitter + 1, size=N), 0, W - 1)
    ys = np.clip(GY[pick] + rng.integers(-jitter, jitter + 1, size=N), 0, H - 1)
    # jitter < spacing / 2 keeps grid points distinct; clipping at the border
    # can only merge points that were already distinct columns/rows apart.
    return xs.astype(np.int64), ys.astype(np.int64)


# ----------------------------------------------------------------------------
# generators
# ----------------------------------------------------------------------------

def make_polygon_pair(H, W, n_regions, seed, *, N, K, a=1.0,
                      strength=(0.5, 1.0), sigma=0.02, t_range=20.0,
                      lin_range=0.05, noise_sd=0.5, outlier_frac=0.05,
                      outlier_R=None, strips=False, grid=False,
                      name="") -> Pair:
    """Random convex polygon regions (and optionally thin rotated strips)
    painted in order over a background, each with its own affine motion."""
    rng = np.random.Generator(np.random.PCG64(seed))
    R = np.zeros((H, W), dtype=np.int32)
    n_strips = n_regions // 4 if strips else 0
    for rid in range(1, n_regions + 1):
        if rid > n_regions - n_strips:
            # thin occluding strip: rotated rectangle, width 8-30 px
            width = rng.uniform(8.0, 30.0)
            length = rng.uniform(0.2, 0.6) * max(H, W)
            ang = rng.uniform(0.0, math.pi)
            cx, cy = rng.uniform(0, W), rng.uniform(0, H)
            d = np.array([math.cos(ang), math.sin(ang)])
            nrm = np.array([-d[1], d[0]])
            c = np.array([cx, cy])
            pts = np.array([c + 0.5 * length * d + 0.5 * width * nrm,
                            c - 0.5 * length * d + 0.5 * width * nrm,
                            c - 0.5 * length * d - 0.5 * width * nrm,
                            c + 0.5 * length * d - 0.5 * width * nrm])
        else:
            bw = rng.uniform(0.15, 0.5) * W
            bh = rng.uniform(0.15, 0.5) * H
            bx = rng.uniform(-0.1 * W, W - 0.9 * bw)
            by = rng.uniform(-0.1 * H, H - 0.9 * bh)
            k = int(rng.integers(5, 9))
            pts = np.stack([rng.uniform(bx, bx + bw, size=k),
                            rng.uniform(by, by + bh, size=k)], axis=1)
        _paint_convex(R, _hull(pts), rid)
    strength_r = rng.uniform(strength[0], strength[1], size=n_regions + 1)
    E = _boundary_strength(R, strength_r)
    C = _cost_from_edges(rng, E, sigma)
    motions = [_region_motion(rng, R, rid, t_range, lin_range)
               for rid in range(n_regions + 1)]
    gt = _affine_flow(R, motions)
    if grid:
        xs, ys = _jittered_grid(rng, H, W, N)
    else:
        flat = rng.choice(H * W, N, replace=False)
        xs, ys = flat % W, flat // W
    m = _make_matches(rng, gt, xs, ys, noise_sd, outlier_frac,
                      t_range if outlier_R is None else outlier_R)
    return Pair(H, W, C, m, gt.astype(np.float32), K, a, name, R)


def make_kitti_pair(H, W, seed, *, N=8000, K=100, a=1.0, n_boxes=20,
                    max_flow=120.0, sigma=0.02, noise_sd=0.5,
                    outlier_frac=0.08, name="") -> Pair:
    """Driving-scene shape: a ground plane below the horizon y_h = H/3 whose
    flow grows linearly toward the bottom rows (expansion about the focus of
    expansion (W/2, y_h)), 20 axis-aligned boxes with independent affine
    motions, and weak texture edges inside regions."""
    rng = np.random.Generator(np.random.PCG64(seed))
    y_h = H / 3.0
    R = np.zeros((H, W), dtype=np.int32)          # 0 = sky
    R[int(math.ceil(y_h)):, :] = 1                # 1 = ground plane
    for b in range(n_boxes):
        bw = rng.uniform(30, 200)
        bh = rng.uniform(20, 120)
        x0 = rng.uniform(0, W - bw)
        ybot = rng.uniform(y_h + 10, H)
        y0 = max(ybot - bh, 0.0)
        R[int(y0):int(ybot), int(x0):int(x0 + bw)] = 2 + b
    n_regions = n_boxes + 2
    strength_r = rng.uniform(0.5, 1.0, size=n_regions)
    E = _boundary_strength(R, strength_r)
    # texture segments inside regions (strength 0.05-0.3), 2 px wide
    for _ in range(int(H * W / 1500)):
        x, y = rng.uniform(0, W), rng.uniform(0, H)
        ang = rng.uniform(0, math.pi)
        ln = rng.uniform(5, 40)
        s = rng.uniform(0.05, 0.3)
        ts = np.linspace(0, ln, int(ln * 2) + 2)
        px = np.clip(np.round(x + ts * math.cos(ang)).astype(int), 0, W - 1)
        py = np.clip(np.round(y + ts * math.sin(ang)).astype(int), 0, H - 1)
        for ox, oy in ((0, 0), (1, 0), (0, 1), (1, 1)):
            qx = np.clip(px + ox, 0, W - 1)
            qy = np.clip(py + oy, 0, H - 1)
            E[qy, qx] = np.maximum(E[qy, qx], s)
    C = _cost_from_edges(rng, E, sigma)

    ys, xs = np.mgrid[0:H, 0:W].astype(np.float64)
    flow = np.zeros((H, W, 2))
    ground = R == 1
    fx, fy = W / 2.0, y_h
    sc = np.clip((ys - y_h) / (H - y_h), 0.0, None)
    mag = sc * np.hypot(xs - fx, ys - fy)
    kappa = max_flow / max(mag[ground].max(), 1e-9)
    flow[..., 0] = np.where(ground, kappa * sc * (xs - fx), 0.0)
    flow[..., 1] = np.where(ground, kappa * sc * (ys - fy), 0.0)
    sky_t = rng.uniform(-2.0, 2.0, size=2)
    flow[R == 0, 0] = sky_t[0]
    flow[R == 0, 1] = sky_t[1]
    for b in range(n_boxes):
        rid = 2 + b
        m = R == rid
        if not m.any():
            continue
        c, A, t = _region_motion(rng, R, rid, 60.0, 0.05)
        dx = xs[m] - c[0]
        dy = ys[m] - c[1]
        flow[m, 0] = c[0] + A[0, 0] * dx + A[0, 1] * dy + t[0] - xs[m]
        flow[m, 1] = c[1] + A[1, 0] * dx + A[1, 1] * dy + t[1] - ys[m]

    # ~90% of the matches in the lower two thirds
    top = int(math.ceil(y_h))
    n_low = int(round(0.9 * N))
    n_top = N - n_low
    low = rng.choice((H - top) * W, n_low, replace=False) + top * W
    hi = rng.choice(top * W, n_top, replace=False)
    flat = np.concatenate([low, hi])
    m = _make_matches(rng, flow, flat % W, flat // W, noise_sd, outlier_frac,
                      max_flow)
    return Pair(H, W, C, m, flow.astype(np.float32), K, a, name, R)


_BATCH_SIZES = ((480, 640), (436, 1024), (375, 1242), (1080, 1920))
_SERVE_SIZES = ((480, 640), (436, 1024), (375, 1242), (1024, 2048))


def config_pair(config: int, index: int = 0) -> Pair:
    """Pair `index` of configuration `config` (1..5); seed 1000*config+index."""
    seed = 1000 * config + index
    if config == 1:
        return make_polygon_pair(128, 256, 6, seed, N=500, K=32, a=1.0,
                                 strength=(0.5, 1.0), sigma=0.02,
                                 t_range=20.0, lin_range=0.05,
                                 noise_sd=0.5, outlier_frac=0.05,
                                 name=CONFIG_NAMES[1])
    if config == 2:
        return make_polygon_pair(436, 1024, 40, seed, N=5000, K=100, a=1.0,
                                 strength=(0.2, 1.0), sigma=0.02,
                                 t_range=150.0, lin_range=0.05,
                                 noise_sd=0.5, outlier_frac=0.10,
                                 strips=True, grid=True,
                                 name=CONFIG_NAMES[2])
    if config == 3:
        return make_kitti_pair(375, 1242, seed, N=8000, K=100, a=1.0,
                               name=CONFIG_NAMES[3])
    if config == 4:
        rng = np.random.Generator(np.random.PCG64(seed))
        H, W = _BATCH_SIZES[int(rng.integers(0, len(_BATCH_SIZES)))]
        N = int(np.clip(round(H * W / 100), 2000, 20000))
        K = int((64, 100, 128)[int(rng.integers(0, 3))])
        nreg = int(rng.integers(10, 81))
        return make_polygon_pair(H, W, nreg, seed + 500_000, N=N, K=K,
                                 a=1.0, strength=(0.2, 1.0), sigma=0.02,
                                 t_range=150.0, lin_range=0.05,
                                 noise_sd=0.5, outlier_frac=0.10,
                                 strips=True, grid=True,
                                 name=CONFIG_NAMES[4])
    if config == 5:
        rng = np.random.Generator(np.random.PCG64(seed))
        H, W = _SERVE_SIZES[int(rng.integers(0, len(_SERVE_SIZES)))]
        N = int(min(H * W / 100 * rng.uniform(0.7, 1.4), 30000))
        nreg = int(rng.integers(10, 81))
        return make_polygon_pair(H, W, nreg, seed + 500_000, N=N, K=100,
                                 a=1.0, strength=(0.2, 1.0), sigma=0.02,
                                 t_range=150.0, lin_range=0.05,
                                 noise_sd=0.5, outlier_frac=0.10,
                                 strips=True, grid=True,
                                 name=CONFIG_NAMES[5])
    raise ValueError(f"unknown config {config}")


def batch_pairs(n: int = 64, config: int = 4):
    """The pairs of a batched launch (config 4 draws mixed sizes)."""
    return [config_pair(config, i) for i in range(n)]


def serving_requests(n: int, rate_hz: float, seed: int = 5000):
    """Poisson arrival times (seconds) for n requests at the given rate; the
    i-th request's pair is config_pair(5, i)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    gaps = rng.exponential(1.0 / rate_hz, size=n)
    return np.cumsum(gaps) - gaps[0]


def region_image(pair: Pair, seed: int = 0, channels: int = 3) -> np.ndarray:
    """A synthetic image float32 [H, W, channels] in [0, 1] of the pair's
    first frame: a random colour per region, a texture of three random plane
    waves per region (so that brightness constancy pins the motion inside a
    region, as texture does in real frames) and pixel noise; the image
    gradient is strongest at region boundaries."""
    if pair.regions is None:
        raise ValueError("pair has no region map")
    R = pair.regions
    H, W = R.shape
    rng = np.random.Generator(np.random.PCG64(seed))
    nreg = int(R.max()) + 1
    base = rng.uniform(0.15, 0.85, size=(nreg, channels))
    ys, xs = np.mgrid[0:H, 0:W].astype(np.float64)
    img = base[R].astype(np.float64)
    for _ in range(3):
        ang = rng.uniform(0, math.pi, size=nreg)
        freq = rng.uniform(0.1, 0.5, size=nreg)
        amp = rng.uniform(0.03, 0.08, size=nreg)
        phase = rng.uniform(0, 2 * math.pi, size=nreg)
        wave = amp[R] * np.sin(freq[R] * (np.cos(ang[R]) * xs + np.sin(ang[R]) * ys) + phase[R])
        img += wave[..., None]
    img += rng.normal(0.0, 0.005, size=img.shape)
    return np.clip(img, 0.0, 1.0).astype(np.float32)


def _bilinear(img: np.ndarray, X: np.ndarray, Y: np.ndarray) -> np.ndarray:
    """img [H, W, ...] sampled at (X, Y), coordinates clamped to the image."""
    H, W = img.shape[:2]
    X = np.clip(X, 0, W - 1)
    Y = np.clip(Y, 0, H - 1)
    x0 = np.minimum(np.floor(X).astype(np.int64), max(W - 2, 0))
    y0 = np.minimum(np.floor(Y).astype(np.int64), max(H - 2, 0))
    x1 = np.minimum(x0 + 1, W - 1)
    y1 = np.minimum(y0 + 1, H - 1)
    ax = (X - x0)[..., None]
    ay = (Y - y0)[..., None]
    I = img.astype(np.float64)
    return ((1 - ay) * ((1 - ax) * I[y0, x0] + ax * I[y0, x1]) +
            ay * ((1 - ax) * I[y1, x0] + ax * I[y1, x1]))


def second_frame(image: np.ndarray, flow: np.ndarray, iterations: int = 12) -> np.ndarray:
    """A second frame for `image` under the forward flow `flow` [H, W, 2]
    (pixel p moves to p + u(p)): I2(q) = I1(q - v(q)), where the backward flow
    v solves v(q) = u(q - v(q)) by fixed-point iteration (bilinear samples of
    u).  Then I2(p + u(p)) = I1(p) wherever the motion is smooth and the
    target is visible; at motion boundaries (occlusions) the iteration takes
    whichever side it settles on.  For a translation v = u after one step."""
    H, W = image.shape[:2]
    ys, xs = np.mgrid[0:H, 0:W].astype(np.float64)
    u = flow.astype(np.float64)
    v = u.copy()
    for _ in range(iterations):
        v = _bilinear(u, xs - v[..., 0], ys - v[..., 1])
    out = _bilinear(image, xs - v[..., 0], ys - v[..., 1])
    return out.astype(np.float32)


def smooth_perturbation(H: int, W: int, rms: float, seed: int = 0,
                        scale: int = 32) -> np.ndarray:
    """A smooth random flow field float32 [H, W, 2] with the given RMS
    magnitude: Gaussian values on a grid of `scale`-pixel spacing,
    interpolated bilinearly."""
    rng = np.random.Generator(np.random.PCG64(seed))
    gh, gw = H // scale + 2, W // scale + 2
    g = rng.normal(size=(gh, gw, 2))
    ys, xs = np.mgrid[0:H, 0:W].astype(np.float64)
    f = _bilinear(g, xs / scale, ys / scale)
    f *= rms / np.sqrt((f ** 2).sum(-1).mean())
    return f.astype(np.float32)


def in_frame(flow: np.ndarray) -> np.ndarray:
    """bool [H, W]: pixels whose target p + u(p) lies inside the frame."""
    H, W = flow.shape[:2]
    ys, xs = np.mgrid[0:H, 0:W].astype(np.float64)
    tx, ty = xs + flow[..., 0], ys + flow[..., 1]
    return (tx >= 0) & (tx <= W - 1) & (ty >= 0) & (ty <= H - 1)
