"""FP64 CPU oracle for the EpicFlow sparse-to-dense interpolator.

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg are the only callers.  The library and its
Python binding never import this package; it shares no code with them.

The arithmetic lives in ``epic_oracle.c`` (plain C, FP64, one thread per
call); this module compiles it with gcc on first use and wraps each step with
numpy arrays.  Functions follow the paper's Algorithm 1 (LA form, Sec. 3.4):

  geodesic(C, matches)            -> D, L      assignment map (Sec. 3.4, Eq. 3)
  graph(C, D, L, matches)         -> em, en, ew    match graph G (Sec. 3.4)
  knn(N, em, en, ew, K)           -> idx, dist, count   N_K by Dijkstra on G
  fit(matches, idx, dist, count, a)  -> model, fallback, detratio  (Eq. 2)
  writeout(L, matches, model)     -> flow      (Algorithm 1, steps 7-8)
  nw(matches, idx, dist, count, a)   -> Nadaraya-Watson flow estimate (Eq. 1)
  interp(C, matches, K, a)        -> dict with every intermediate
  consistency(C, matches, a, ...) -> keep flags of the NW consistency check
                                     (Sec. 4.1, "Pruning of matches")
  interp_pruned(C, matches, K, a) -> the check, then interp on the kept matches
  gradient_cost(image)            -> the ||grad I|| cost map of Table 2
  refine.refine(I1, I2, flow)     -> the variational refinement of Sec. 4
                                     (module oracle/refine.py, numpy)
  interp_exact(C, matches, K, a)  -> the exact variant of Sec. 5.2: distances
                                     from every pixel to every match and a fit
                                     per pixel (geodesic or Euclidean)

Parity status of each function and the pins that check it are listed in the
test files ``tests/test_oracle_*.py``; every function here is pinned.
"""

from __future__ import annotations

import ctypes
import os
import platform
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "epic_oracle.c")
_BUILD = os.path.join(_HERE, "_build", platform.machine() or "unknown")
_LIB = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

ORACLE_OK = 0


def build(force: bool = False) -> str:
    """Compile the oracle shared library (gcc, -O2, no FP contraction)."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    subprocess.check_call([
        "gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off",
        "-Wall", "-Wextra", "-Wno-unused-parameter", "-o", tmp, _SRC, "-lm",
    ])
    os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        build()
        lib = ctypes.CDLL(_LIB)
        P = ctypes.c_void_p
        I = ctypes.c_int
        Lg = ctypes.c_long
        D = ctypes.c_double
        lib.epic_oracle_geodesic.argtypes = [P, I, I, P, I, P, P]
        lib.epic_oracle_geodesic.restype = I
        lib.epic_oracle_graph.argtypes = [P, I, I, P, P, P, I, P, P, P, Lg]
        lib.epic_oracle_graph.restype = Lg
        lib.epic_oracle_knn.argtypes = [I, Lg, P, P, P, I, P, P, P]
        lib.epic_oracle_knn.restype = I
        lib.epic_oracle_fit.argtypes = [I, P, I, P, P, P, D, I, P, P, P]
        lib.epic_oracle_fit.restype = I
        lib.epic_oracle_writeout.argtypes = [I, I, P, I, P, P, P]
        lib.epic_oracle_writeout.restype = I
        lib.epic_oracle_nw.argtypes = [I, P, I, P, P, P, D, P]
        lib.epic_oracle_nw.restype = I
        lib.epic_oracle_fit_points.argtypes = [I, P, I, P, I, P, P, P, D, I, P, P, P]
        lib.epic_oracle_fit_points.restype = I
        _lib = lib
        return lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _check(rc, what):
    if rc != ORACLE_OK:
        raise RuntimeError(f"oracle {what} failed with code {rc}")


def _f32(a):
    return np.ascontiguousarray(a, dtype=np.float32)


def geodesic(C, matches):
    """D float64 [H, W], L int32 [H, W] (Sec. 3.4 assignment, Eq. 3)."""
    lib = _load()
    C = _f32(C)
    matches = _f32(matches).reshape(-1, 4)
    H, W = C.shape
    D = np.empty((H, W), np.float64)
    L = np.empty((H, W), np.int32)
    _check(lib.epic_oracle_geodesic(_ptr(C), H, W, _ptr(matches),
                                    matches.shape[0], _ptr(D), _ptr(L)),
           "geodesic")
    return D, L


def graph(C, D, L, matches):
    """Edges (em < en, ew) of G sorted by (em, en)."""
    lib = _load()
    C = _f32(C)
    H, W = C.shape
    D = np.ascontiguousarray(D, np.float64)
    L = np.ascontiguousarray(L, np.int32)
    matches = _f32(matches).reshape(-1, 4)
    N = matches.shape[0]
    cap = 4 * H * W + N + 1
    em = np.empty(cap, np.int32)
    en = np.empty(cap, np.int32)
    ew = np.empty(cap, np.float64)
    ne = lib.epic_oracle_graph(_ptr(C), H, W, _ptr(D), _ptr(L), _ptr(matches),
                               N, _ptr(em), _ptr(en), _ptr(ew), cap)
    if ne < 0:
        raise RuntimeError(f"oracle graph failed with code {ne}")
    return em[:ne].copy(), en[:ne].copy(), ew[:ne].copy()


def knn(N, em, en, ew, K):
    """idx int32 [N, K], dist float64 [N, K], count int32 [N]."""
    lib = _load()
    em = np.ascontiguousarray(em, np.int32)
    en = np.ascontiguousarray(en, np.int32)
    ew = np.ascontiguousarray(ew, np.float64)
    idx = np.full((N, K), -1, np.int32)
    dist = np.full((N, K), np.inf, np.float64)
    count = np.zeros(N, np.int32)
    _check(lib.epic_oracle_knn(N, len(em), _ptr(em), _ptr(en), _ptr(ew), K,
                               _ptr(idx), _ptr(dist), _ptr(count)), "knn")
    return idx, dist, count


def fit(matches, idx, dist, count, a, weight_squared=True):
    """model float64 [N, 6] = (c_u, c_v, b11, b12, b21, b22), fallback int32
    [N], detratio float64 [N]."""
    lib = _load()
    matches = _f32(matches).reshape(-1, 4)
    N = matches.shape[0]
    idx = np.ascontiguousarray(idx, np.int32)
    dist = np.ascontiguousarray(dist, np.float64)
    count = np.ascontiguousarray(count, np.int32)
    K = idx.shape[1]
    model = np.empty((N, 6), np.float64)
    fb = np.empty(N, np.int32)
    dr = np.empty(N, np.float64)
    _check(lib.epic_oracle_fit(N, _ptr(matches), K, _ptr(idx), _ptr(dist),
                               _ptr(count), float(a), int(bool(weight_squared)),
                               _ptr(model), _ptr(fb), _ptr(dr)), "fit")
    return model, fb, dr


def writeout(L, matches, model):
    """flow float64 [H, W, 2] = c_L + B_L (p - p_L)."""
    lib = _load()
    L = np.ascontiguousarray(L, np.int32)
    H, W = L.shape
    matches = _f32(matches).reshape(-1, 4)
    model = np.ascontiguousarray(model, np.float64)
    flow = np.empty((H, W, 2), np.float64)
    _check(lib.epic_oracle_writeout(H, W, _ptr(L), matches.shape[0],
                                    _ptr(matches), _ptr(model), _ptr(flow)),
           "writeout")
    return flow


def nw(matches, idx, dist, count, a):
    """Nadaraya-Watson estimate at every match, float64 [N, 2]: the
    kernel-weighted mean of the neighbours' flows p'_n - p_n (Eq. 1)."""
    lib = _load()
    matches = _f32(matches).reshape(-1, 4)
    N = matches.shape[0]
    idx = np.ascontiguousarray(idx, np.int32)
    dist = np.ascontiguousarray(dist, np.float64)
    count = np.ascontiguousarray(count, np.int32)
    out = np.empty((N, 2), np.float64)
    _check(lib.epic_oracle_nw(N, _ptr(matches), idx.shape[1], _ptr(idx),
                              _ptr(dist), _ptr(count), float(a), _ptr(out)),
           "nw")
    return out


def interp(C, matches, K, a, weight_squared=True, estimator="la"):
    """The whole interpolator (Algorithm 1) with every intermediate.

    estimator "la": locally-weighted affine fit per match (Eq. 2, with the
    NW fallback of a degenerate fit); "nw": the Nadaraya-Watson flow of
    Eq. 1 per match, constant over the match's cell (Algorithm 1)."""
    matches = _f32(matches).reshape(-1, 4)
    N = matches.shape[0]
    K = int(min(K, N))
    D, L = geodesic(C, matches)
    em, en, ew = graph(C, D, L, matches)
    idx, dist, count = knn(N, em, en, ew, K)
    if estimator == "la":
        model, fb, dr = fit(matches, idx, dist, count, a, weight_squared)
    elif estimator == "nw":
        model = np.zeros((N, 6), np.float64)
        model[:, :2] = nw(matches, idx, dist, count, a)
        fb = np.ones(N, np.int32)
        dr = np.zeros(N, np.float64)
    else:
        raise ValueError(f"unknown estimator {estimator!r}")
    flow = writeout(L, matches, model)
    return dict(D=D, L=L, em=em, en=en, ew=ew, idx=idx, dist=dist,
                count=count, model=model, fallback=fb, detratio=dr,
                flow=flow, K=K)


def consistency(C, matches, a, threshold=5.0, K_nw=25):
    """Consistency check of Sec. 4.1 ("Pruning of matches"): the NW
    interpolation is run once on all matches (K_nw neighbours, Eq. 1) and a
    match is kept when the Euclidean distance between its own flow
    p'_m - p_m and the estimate at p_m is at most `threshold` px.

    Returns (keep bool [N], deviation float64 [N], the NW run's dict)."""
    matches = _f32(matches).reshape(-1, 4)
    r = interp(C, matches, K_nw, a, estimator="nw")
    own = matches[:, 2:].astype(np.float64) - matches[:, :2].astype(np.float64)
    dev = np.hypot(*(r["model"][:, :2] - own).T)
    return dev <= threshold, dev, r


def interp_pruned(C, matches, K, a, threshold=5.0, K_nw=25, weight_squared=True,
                  estimator="la"):
    """Consistency check, then the interpolator on the kept matches.  When
    no match passes, all are kept.  The result dict adds keep (flags over
    the submitted matches), kept_index (original index of every match used)
    and deviation."""
    matches = _f32(matches).reshape(-1, 4)
    keep, dev, _ = consistency(C, matches, a, threshold, K_nw)
    kept_index = np.flatnonzero(keep) if keep.any() else np.arange(matches.shape[0])
    r = interp(C, matches[kept_index], K, a, weight_squared, estimator)
    r.update(keep=keep, kept_index=kept_index.astype(np.int32), deviation=dev)
    return r


def fit_points(centres, matches, idx, dist, count, a, weight_squared=True):
    """Fit of Eq. 2 centred at arbitrary points: model float64 [Np, 6]
    (flow at the centre = model[:, :2]), fallback int32 [Np], detratio."""
    lib = _load()
    centres = np.ascontiguousarray(centres, np.float64).reshape(-1, 2)
    matches = _f32(matches).reshape(-1, 4)
    idx = np.ascontiguousarray(idx, np.int32)
    dist = np.ascontiguousarray(dist, np.float64)
    count = np.ascontiguousarray(count, np.int32)
    Np, K = idx.shape
    model = np.empty((Np, 6), np.float64)
    fb = np.empty(Np, np.int32)
    dr = np.empty(Np, np.float64)
    _check(lib.epic_oracle_fit_points(Np, _ptr(centres), matches.shape[0], _ptr(matches), K,
                                      _ptr(idx), _ptr(dist), _ptr(count), float(a),
                                      int(bool(weight_squared)), _ptr(model), _ptr(fb),
                                      _ptr(dr)), "fit_points")
    return model, fb, dr


def exact_distances(C, matches, metric="geodesic"):
    """float64 [N, H, W]: distance from every pixel to every match.

    "geodesic": D_G of Eq. 3, one single-source transform per match (the
    multi-source transform run on that match alone); "euclidean": the
    distance between pixel centres and the match's source pixel."""
    matches = _f32(matches).reshape(-1, 4)
    C = _f32(C)
    H, W = C.shape
    N = matches.shape[0]
    out = np.empty((N, H, W), np.float64)
    if metric == "geodesic":
        for m in range(N):
            out[m], _ = geodesic(C, matches[m:m + 1])
    elif metric == "euclidean":
        ys, xs = np.mgrid[0:H, 0:W].astype(np.float64)
        sx = np.floor(matches[:, 0].astype(np.float64) + 0.5)
        sy = np.floor(matches[:, 1].astype(np.float64) + 0.5)
        for m in range(N):
            out[m] = np.hypot(xs - sx[m], ys - sy[m])
    else:
        raise ValueError(f"unknown metric {metric!r}")
    return out


def interp_exact(C, matches, K, a, metric="geodesic", weight_squared=True,
                 estimator="la"):
    """Exact variant (Sec. 5.2, Table 2): every pixel p takes its own K
    nearest matches under the exact distance (key (d, index)) and its own
    fit (Eq. 2 centred at p, or the NW estimate of Eq. 1); the flow at p is
    the model's value at its centre."""
    matches = _f32(matches).reshape(-1, 4)
    H, W = np.asarray(C).shape
    N = matches.shape[0]
    K = int(min(K, N))
    Dall = exact_distances(C, matches, metric).reshape(N, -1)
    P = H * W
    idx = np.empty((P, K), np.int32)
    dist = np.empty((P, K), np.float64)
    order = np.arange(N)
    for p in range(P):
        sel = np.lexsort((order, Dall[:, p]))[:K]   # by distance, then index
        idx[p] = sel
        dist[p] = Dall[sel, p]
    count = np.full(P, K, np.int32)
    ys, xs = np.mgrid[0:H, 0:W]
    centres = np.stack([xs.ravel(), ys.ravel()], 1).astype(np.float64)
    if estimator == "la":
        model, fb, dr = fit_points(centres, matches, idx, dist, count, a, weight_squared)
    elif estimator == "nw":
        k = np.exp(-a * dist)
        u = (matches[idx, 2].astype(np.float64) - matches[idx, 0])
        v = (matches[idx, 3].astype(np.float64) - matches[idx, 1])
        model = np.zeros((P, 6))
        model[:, 0] = (k * u).sum(1) / k.sum(1)
        model[:, 1] = (k * v).sum(1) / k.sum(1)
        fb, dr = np.ones(P, np.int32), np.zeros(P)
    else:
        raise ValueError(f"unknown estimator {estimator!r}")
    flow = model[:, :2].reshape(H, W, 2).copy()
    return dict(flow=flow, idx=idx, dist=dist, count=count, model=model,
                fallback=fb, detratio=dr, K=K)


def gradient_cost(image, floor=0.0):
    """Cost map from the image gradient (Table 2, the "||grad_2 I||_2"
    contour row): C(p) = floor + sqrt(sum over channels of gx^2 + gy^2),
    with central differences gx = (I(x+1) - I(x-1)) / 2 on the image padded
    by edge replication (so gx = (I(1) - I(0)) / 2 at the left border).
    image: [H, W] or [H, W, channels], values in [0, 1]; float64 [H, W] out."""
    I = np.asarray(image, np.float64)
    if I.ndim == 2:
        I = I[..., None]
    Ip = np.pad(I, ((1, 1), (1, 1), (0, 0)), mode="edge")
    gx = (Ip[1:-1, 2:] - Ip[1:-1, :-2]) / 2.0
    gy = (Ip[2:, 1:-1] - Ip[:-2, 1:-1]) / 2.0
    return floor + np.sqrt((gx * gx + gy * gy).sum(axis=2))
