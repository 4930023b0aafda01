"""ctypes binding of ``libepic_interp.so`` (declared in include/epic_interp.h).

Argument marshalling only: every step of the interpolator runs in the CUDA
library.  Function names mirror the C ABI; ``EpicInterp`` is a small
convenience wrapper that takes torch CUDA tensors for device buffers and the
current torch stream.  Importing raises if the library has not been built
(``python -m paper_1501_02565_gb300.build``); there is no CPU fallback.
"""

from __future__ import annotations

import ctypes
import os

from . import build as _build

EPIC_OK = 0
EPIC_ERR_INVALID = 1
EPIC_ERR_OOM = 2
EPIC_ERR_CUDA = 3
EPIC_ERR_NOT_CONVERGED = 4
EPIC_ERR_TIMEOUT = 5
EPIC_ERR_CAPACITY = 6
EPIC_MAX_K = 2048

STATUS_NAMES = {
    0: "EPIC_OK", 1: "EPIC_ERR_INVALID", 2: "EPIC_ERR_OOM", 3: "EPIC_ERR_CUDA",
    4: "EPIC_ERR_NOT_CONVERGED", 5: "EPIC_ERR_TIMEOUT", 6: "EPIC_ERR_CAPACITY",
}

# Every symbol include/epic_interp.h declares.
EXPORTED = (
    "epic_config_default", "epic_interp_create", "epic_interp_run",
    "epic_interp_run_batch", "epic_interp_run_host",
    "epic_interp_run_batch_host", "epic_interp_submit_batch_host", "epic_interp_sync",
    "epic_interp_get_labels", "epic_interp_get_edge_count",
    "epic_interp_get_graph", "epic_interp_get_knn", "epic_interp_get_models",
    "epic_interp_get_pruning", "epic_interp_get_passes", "epic_interp_get_knn_retries",
    "epic_interp_get_distance_unit",
    "epic_interp_set_tile_rules",
    "epic_interp_enable_stage_timing",
    "epic_interp_get_stage_times", "epic_interp_request_bytes",
    "epic_interp_launches_per_run",
    "epic_interp_last_error", "epic_interp_destroy",
    "epic_geodesic_labels_noalloc", "epic_exact_interp", "epic_gradient_cost",
    "epic_refine_params_default", "epic_refine", "epic_selftest_wait_timeout",
)


class epic_config_t(ctypes.Structure):
    _fields_ = [
        ("max_H", ctypes.c_int), ("max_W", ctypes.c_int),
        ("max_N", ctypes.c_int), ("max_K", ctypes.c_int),
        ("max_pairs", ctypes.c_int), ("max_passes", ctypes.c_int),
        ("weight_squared", ctypes.c_int), ("fallback_eps", ctypes.c_float),
        ("tile_w", ctypes.c_int), ("tile_h", ctypes.c_int),
        ("apron", ctypes.c_int), ("keep_intermediates", ctypes.c_int),
        ("max_degree", ctypes.c_int), ("use_graphs", ctypes.c_int),
        ("estimator", ctypes.c_int), ("prune", ctypes.c_int),
        ("prune_threshold", ctypes.c_float), ("prune_K", ctypes.c_int),
        ("sweep", ctypes.c_int), ("exact_chunk_bytes", ctypes.c_longlong),
    ]


class epic_refine_params_t(ctypes.Structure):
    _fields_ = [
        ("alpha0", ctypes.c_float), ("gamma", ctypes.c_float), ("kappa", ctypes.c_float),
        ("eps", ctypes.c_float), ("zeta", ctypes.c_float), ("omega", ctypes.c_float),
        ("iterations", ctypes.c_int), ("sor_iterations", ctypes.c_int),
    ]


class epic_pair_desc_t(ctypes.Structure):
    _fields_ = [
        ("cost_map", ctypes.c_void_p), ("matches", ctypes.c_void_p),
        ("H", ctypes.c_int), ("W", ctypes.c_int), ("N", ctypes.c_int),
        ("K", ctypes.c_int), ("a", ctypes.c_float),
        ("flow_out", ctypes.c_void_p),
    ]


class epic_tile_rule_t(ctypes.Structure):
    _fields_ = [
        ("max_pixels", ctypes.c_longlong), ("tile_w", ctypes.c_int),
        ("tile_h", ctypes.c_int), ("apron", ctypes.c_int), ("sweep", ctypes.c_int),
    ]


class EpicError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{STATUS_NAMES.get(code, code)}: {msg}")
        self.code = code


_lib = None


def library_path() -> str:
    return _build.LIB


def load(path: str | None = None):
    """Load the shared library (raises OSError if it is missing)."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or _build.LIB
    if not os.path.exists(path):
        raise OSError(
            f"{path} not found: build it with `python -m paper_1501_02565_gb300.build`")
    lib = ctypes.CDLL(path)
    P, I, F = ctypes.c_void_p, ctypes.c_int, ctypes.c_float
    pp = ctypes.POINTER(ctypes.c_void_p)
    pi = ctypes.POINTER(ctypes.c_int)
    lib.epic_config_default.argtypes = [ctypes.POINTER(epic_config_t)]
    lib.epic_config_default.restype = None
    lib.epic_interp_create.argtypes = [pp, I, ctypes.POINTER(epic_config_t)]
    lib.epic_interp_create.restype = I
    lib.epic_interp_run.argtypes = [P, P, P, I, I, I, I, F, P, P]
    lib.epic_interp_run.restype = I
    lib.epic_interp_run_batch.argtypes = [P, ctypes.POINTER(epic_pair_desc_t), I, P]
    lib.epic_interp_run_batch.restype = I
    lib.epic_interp_run_host.argtypes = [P, P, P, I, I, I, I, F, P, P]
    lib.epic_interp_run_host.restype = I
    lib.epic_interp_run_batch_host.argtypes = [P, ctypes.POINTER(epic_pair_desc_t), I, P]
    lib.epic_interp_run_batch_host.restype = I
    lib.epic_interp_submit_batch_host.argtypes = [P, ctypes.POINTER(epic_pair_desc_t), I]
    lib.epic_interp_submit_batch_host.restype = I
    lib.epic_interp_sync.argtypes = [P]
    lib.epic_interp_sync.restype = I
    lib.epic_interp_get_labels.argtypes = [P, I, P, P, P]
    lib.epic_interp_get_labels.restype = I
    lib.epic_interp_get_edge_count.argtypes = [P, I, pi]
    lib.epic_interp_get_edge_count.restype = I
    lib.epic_interp_get_graph.argtypes = [P, I, P, P, P, I, pi]
    lib.epic_interp_get_graph.restype = I
    lib.epic_interp_get_knn.argtypes = [P, I, P, P, P, P]
    lib.epic_interp_get_knn.restype = I
    lib.epic_interp_get_models.argtypes = [P, I, P, P, P]
    lib.epic_interp_get_models.restype = I
    lib.epic_interp_get_pruning.argtypes = [P, I, P, P, pi]
    lib.epic_interp_get_pruning.restype = I
    lib.epic_interp_get_passes.argtypes = [P, pi]
    lib.epic_interp_get_passes.restype = I
    lib.epic_interp_get_distance_unit.argtypes = [P, I, pi]
    lib.epic_interp_get_distance_unit.restype = I
    lib.epic_interp_get_knn_retries.argtypes = [P, pi]
    lib.epic_interp_get_knn_retries.restype = I
    lib.epic_interp_set_tile_rules.argtypes = [P, ctypes.POINTER(epic_tile_rule_t), I]
    lib.epic_interp_set_tile_rules.restype = I
    lib.epic_interp_enable_stage_timing.argtypes = [P, I]
    lib.epic_interp_enable_stage_timing.restype = I
    lib.epic_interp_get_stage_times.argtypes = [P, ctypes.POINTER(ctypes.c_float), I, pi]
    lib.epic_interp_get_stage_times.restype = I
    lib.epic_interp_request_bytes.argtypes = [P, ctypes.POINTER(epic_config_t), I, I, I, I,
                                              ctypes.POINTER(ctypes.c_longlong)]
    lib.epic_interp_request_bytes.restype = I
    lib.epic_interp_launches_per_run.argtypes = [P, I]
    lib.epic_interp_launches_per_run.restype = I
    lib.epic_interp_last_error.argtypes = [P]
    lib.epic_interp_last_error.restype = ctypes.c_char_p
    lib.epic_interp_destroy.argtypes = [P]
    lib.epic_interp_destroy.restype = None
    lib.epic_refine_params_default.argtypes = [ctypes.POINTER(epic_refine_params_t)]
    lib.epic_refine_params_default.restype = None
    lib.epic_refine.argtypes = [P, P, P, I, I, I, P, ctypes.POINTER(epic_refine_params_t), P]
    lib.epic_refine.restype = I
    lib.epic_selftest_wait_timeout.argtypes = [P, I, I]
    lib.epic_selftest_wait_timeout.restype = I
    lib.epic_gradient_cost.argtypes = [P, I, I, I, I, F, P, P]
    lib.epic_gradient_cost.restype = I
    lib.epic_exact_interp.argtypes = [P, P, P, I, I, I, I, F, I, P, P, P, P]
    lib.epic_exact_interp.restype = I
    lib.epic_geodesic_labels_noalloc.argtypes = [P, P, I, I, I, P, P, P]
    lib.epic_geodesic_labels_noalloc.restype = I
    _lib = lib
    return lib


def epic_config_default() -> epic_config_t:
    cfg = epic_config_t()
    load().epic_config_default(ctypes.byref(cfg))
    return cfg


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _stream_handle(stream=None):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


class EpicInterp:
    """Handle over one device; buffers are torch CUDA tensors (float32)."""

    def __init__(self, device: int = 0, **cfg_overrides):
        self.lib = load()
        cfg = epic_config_default()
        for k, v in cfg_overrides.items():
            if not hasattr(cfg, k):
                raise TypeError(f"unknown config field {k}")
            setattr(cfg, k, v)
        self.cfg = cfg
        self.device = device
        h = ctypes.c_void_p()
        rc = self.lib.epic_interp_create(ctypes.byref(h), device, ctypes.byref(cfg))
        if rc != EPIC_OK:
            raise EpicError(rc, "epic_interp_create failed")
        self.h = h
        self._inflight = []   # host tensors of submitted batches, until sync()

    # -- helpers -------------------------------------------------------------
    def _check(self, rc, what):
        if rc != EPIC_OK:
            msg = self.lib.epic_interp_last_error(self.h)
            raise EpicError(rc, f"{what}: {msg.decode() if msg else ''}")

    def close(self):
        if getattr(self, "h", None):
            self.lib.epic_interp_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- entry points --------------------------------------------------------
    def run(self, C, matches, K, a, flow=None, stream=None):
        """Enqueue one pair; C [H, W], matches [N, 4] float32 CUDA tensors."""
        import torch
        H, W = C.shape
        N = matches.shape[0]
        if flow is None:
            flow = torch.empty((H, W, 2), dtype=torch.float32, device=C.device)
        rc = self.lib.epic_interp_run(self.h, _ptr(C), _ptr(matches), H, W, N,
                                      int(K), float(a), _ptr(flow),
                                      _stream_handle(stream))
        self._check(rc, "epic_interp_run")
        return flow

    def run_batch(self, items, stream=None):
        """items: list of (C, matches, K, a, flow) with CUDA tensors."""
        n = len(items)
        arr = (epic_pair_desc_t * n)()
        for i, (C, M, K, a, F) in enumerate(items):
            arr[i] = epic_pair_desc_t(C.data_ptr(), M.data_ptr(), C.shape[0],
                                      C.shape[1], M.shape[0], int(K), float(a),
                                      F.data_ptr())
        rc = self.lib.epic_interp_run_batch(self.h, arr, n, _stream_handle(stream))
        self._check(rc, "epic_interp_run_batch")

    def run_host(self, C, matches, K, a, flow, stream=None):
        """Host buffers (contiguous float32 numpy arrays or CPU tensors)."""
        def addr(x):
            return ctypes.c_void_p(x.ctypes.data if hasattr(x, "ctypes") else x.data_ptr())
        H, W = C.shape
        rc = self.lib.epic_interp_run_host(self.h, addr(C), addr(matches), H, W,
                                           matches.shape[0], int(K), float(a),
                                           addr(flow), _stream_handle(stream))
        self._check(rc, "epic_interp_run_host")

    def run_batch_host(self, items, stream=None):
        """items: list of (C, matches, K, a, flow) with contiguous float32 CPU
        tensors (pinned for asynchronous copies); waits for completion."""
        n = len(items)
        arr = (epic_pair_desc_t * n)()
        for i, (C, M, K, a, F) in enumerate(items):
            arr[i] = epic_pair_desc_t(C.data_ptr(), M.data_ptr(), C.shape[0],
                                      C.shape[1], M.shape[0], int(K), float(a),
                                      F.data_ptr())
        rc = self.lib.epic_interp_run_batch_host(self.h, arr, n, _stream_handle(stream))
        self._check(rc, "epic_interp_run_batch_host")

    def submit_batch_host(self, items):
        """Streaming form of run_batch_host: enqueues the batch (uploads, run,
        downloads) and returns at once; consecutive calls overlap.  The
        tensors are kept alive here until sync()."""
        n = len(items)
        arr = (epic_pair_desc_t * n)()
        for i, (C, M, K, a, F) in enumerate(items):
            arr[i] = epic_pair_desc_t(C.data_ptr(), M.data_ptr(), C.shape[0],
                                      C.shape[1], M.shape[0], int(K), float(a),
                                      F.data_ptr())
        self._inflight.append(items)
        rc = self.lib.epic_interp_submit_batch_host(self.h, arr, n)
        self._check(rc, "epic_interp_submit_batch_host")

    def sync(self):
        rc = self.lib.epic_interp_sync(self.h)
        self._inflight = []
        self._check(rc, "device status")

    def sync_status(self) -> int:
        rc = self.lib.epic_interp_sync(self.h)
        self._inflight = []
        return rc

    def get_labels(self, pair=0, H=None, W=None, stream=None):
        import torch
        P = self._last_shape(pair, H, W)
        L = torch.empty(P, dtype=torch.int32, device=f"cuda:{self.device}")
        D = torch.empty(P, dtype=torch.float32, device=f"cuda:{self.device}")
        self._check(self.lib.epic_interp_get_labels(self.h, pair, _ptr(L), _ptr(D),
                                                    _stream_handle(stream)),
                    "get_labels")
        return L, D

    def _last_shape(self, pair, H, W):
        if H is None or W is None:
            raise ValueError("pass H and W of the pair")
        return (H, W)

    def get_edge_count(self, pair=0):
        n = ctypes.c_int()
        self._check(self.lib.epic_interp_get_edge_count(self.h, pair, ctypes.byref(n)),
                    "get_edge_count")
        return n.value

    def get_graph(self, pair=0):
        import torch
        n = self.get_edge_count(pair)
        dev = f"cuda:{self.device}"
        em = torch.empty(max(n, 1), dtype=torch.int32, device=dev)
        en = torch.empty_like(em)
        ew = torch.empty(max(n, 1), dtype=torch.float32, device=dev)
        cnt = ctypes.c_int()
        self._check(self.lib.epic_interp_get_graph(self.h, pair, _ptr(em), _ptr(en),
                                                   _ptr(ew), max(n, 1),
                                                   ctypes.byref(cnt)), "get_graph")
        k = cnt.value
        return em[:k], en[:k], ew[:k]

    def get_knn(self, pair, N, K, stream=None):
        import torch
        dev = f"cuda:{self.device}"
        K = min(K, N)
        idx = torch.empty((N, K), dtype=torch.int32, device=dev)
        dist = torch.empty((N, K), dtype=torch.float32, device=dev)
        cnt = torch.empty(N, dtype=torch.int32, device=dev)
        self._check(self.lib.epic_interp_get_knn(self.h, pair, _ptr(idx), _ptr(dist),
                                                 _ptr(cnt), _stream_handle(stream)),
                    "get_knn")
        return idx, dist, cnt

    def get_models(self, pair, N, stream=None):
        import torch
        dev = f"cuda:{self.device}"
        models = torch.empty((N, 8), dtype=torch.float32, device=dev)
        fb = torch.empty(N, dtype=torch.int32, device=dev)
        self._check(self.lib.epic_interp_get_models(self.h, pair, _ptr(models), _ptr(fb),
                                                    _stream_handle(stream)),
                    "get_models")
        return models, fb

    def exact(self, C, matches, K, a, metric="geodesic", with_knn=False, stream=None):
        """Exact per-pixel variant (epic_exact_interp); CUDA tensors in,
        flow [H, W, 2] (and per-pixel K-NN lists) out; waits."""
        import torch
        H, W = C.shape
        N = matches.shape[0]
        Kc = min(int(K), N)
        dev = C.device
        flow = torch.empty((H, W, 2), dtype=torch.float32, device=dev)
        idx = dist = None
        if with_knn:
            idx = torch.empty((H * W, Kc), dtype=torch.int32, device=dev)
            dist = torch.empty((H * W, Kc), dtype=torch.float32, device=dev)
        code = {"geodesic": 0, "euclidean": 1}[metric]
        rc = self.lib.epic_exact_interp(self.h, _ptr(C), _ptr(matches), H, W, N, int(K),
                                        float(a), code, _ptr(flow), _ptr(idx), _ptr(dist),
                                        _stream_handle(stream))
        self._check(rc, "epic_exact_interp")
        return (flow, idx, dist) if with_knn else flow

    def refine(self, I1, I2, flow, stream=None, **params):
        """Variational refinement (epic_refine) of the CUDA tensor flow
        [H, W, 2] in place, between images I1, I2 [H, W] or [H, W, C]
        (float32 CUDA tensors in [0, 1]); keyword overrides of the
        parameters (alpha0, gamma, kappa, eps, zeta, omega, iterations,
        sor_iterations).  Enqueued on `stream`."""
        prm = epic_refine_params_t()
        self.lib.epic_refine_params_default(ctypes.byref(prm))
        for k, v in params.items():
            if not hasattr(prm, k):
                raise TypeError(f"unknown refinement parameter {k}")
            setattr(prm, k, v)
        H, W = I1.shape[:2]
        C = 1 if I1.dim() == 2 else I1.shape[2]
        for t in (I1, I2, flow):
            if not t.is_contiguous():
                raise ValueError("tensors must be contiguous")
        rc = self.lib.epic_refine(self.h, _ptr(I1), _ptr(I2), H, W, C, _ptr(flow),
                                  ctypes.byref(prm), _stream_handle(stream))
        self._check(rc, "epic_refine")
        return flow

    def selftest_wait_timeout(self, which, limit_ms=50):
        """Status recorded by a bounded device wait that never completes
        (0: grid barrier, 1: TMA mbarrier); EPIC_ERR_TIMEOUT expected."""
        return self.lib.epic_selftest_wait_timeout(self.h, int(which), int(limit_ms))

    def get_pruning(self, pair, N):
        """Consistency pruning of the last run's pair (prune = 1): keep
        flags [N] of the submitted matches and the original index of every
        match the interpolation used."""
        import torch
        dev = f"cuda:{self.device}"
        keep = torch.empty(N, dtype=torch.int32, device=dev)
        kept = torch.empty(N, dtype=torch.int32, device=dev)
        n = ctypes.c_int()
        self._check(self.lib.epic_interp_get_pruning(self.h, pair, _ptr(keep), _ptr(kept),
                                                     ctypes.byref(n)), "get_pruning")
        return keep, kept[:n.value]

    def get_passes(self):
        n = ctypes.c_int()
        self._check(self.lib.epic_interp_get_passes(self.h, ctypes.byref(n)), "get_passes")
        return n.value

    def get_distance_unit(self, pair=0):
        """Shift s of the pair's distance unit 2^-(31 - s) in the last run."""
        n = ctypes.c_int()
        self._check(self.lib.epic_interp_get_distance_unit(self.h, pair, ctypes.byref(n)),
                    "get_distance_unit")
        return n.value

    def get_knn_retries(self):
        """Matches of the last run whose K-NN search ran again with large tables."""
        n = ctypes.c_int()
        self._check(self.lib.epic_interp_get_knn_retries(self.h, ctypes.byref(n)),
                    "get_knn_retries")
        return n.value

    STAGES = ("prepare", "relax", "edges", "scatter", "knn_fit", "writeout", "prune")

    def set_tile_rules(self, rules):
        """rules: iterable of (max_pixels, tile_w, tile_h, apron[, sweep])."""
        rules = list(rules)
        arr = (epic_tile_rule_t * max(len(rules), 1))()
        for i, r in enumerate(rules):
            mp, tw, th, ap = r[:4]
            sw = r[4] if len(r) > 4 else 0
            arr[i] = epic_tile_rule_t(int(mp), int(tw), int(th), int(ap), int(sw))
        self._check(self.lib.epic_interp_set_tile_rules(self.h, arr, len(rules)),
                    "set_tile_rules")

    def enable_stage_timing(self, enable=True):
        self._check(self.lib.epic_interp_enable_stage_timing(self.h, int(enable)),
                    "enable_stage_timing")

    def stage_times(self):
        """{stage: summed ms} over the timed runs, and the run count."""
        ns = len(self.STAGES)
        arr = (ctypes.c_float * ns)()
        n = ctypes.c_int()
        self._check(self.lib.epic_interp_get_stage_times(self.h, arr, ns, ctypes.byref(n)),
                    "get_stage_times")
        return dict(zip(self.STAGES, list(arr))), n.value

    def request_bytes(self, H, W, N, K):
        """Arena bytes one H x W pair with N matches and K neighbours takes
        in a batch on this handle (epic_interp_request_bytes)."""
        return request_bytes(H, W, N, K, handle=self.h)

    def launches_per_run(self, n=1):
        return self.lib.epic_interp_launches_per_run(self.h, n)


def request_bytes(H, W, N, K, cfg=None, handle=None):
    """epic_interp_request_bytes: the arena bytes of one pair, from the
    handle's configuration and tile rules, else from `cfg` (an epic_config_t,
    None = defaults) without tile rules.  Needs no device."""
    lib = load()
    out = ctypes.c_longlong()
    rc = lib.epic_interp_request_bytes(handle, None if cfg is None else ctypes.byref(cfg),
                                       int(H), int(W), int(N), int(K), ctypes.byref(out))
    if rc != EPIC_OK:
        raise EpicError(rc, "epic_interp_request_bytes")
    return out.value


def gradient_cost(image, floor=0.0, out=None, stream=None):
    """Image-gradient cost map (epic_gradient_cost) of a CUDA float32 tensor
    [H, W], [H, W, channels] or [frames, H, W, channels]; returns [H, W]
    (or [frames, H, W]), enqueued on `stream`."""
    import torch
    lib = load()
    x = image
    if x.dim() == 2:
        x = x[None, :, :, None]
    elif x.dim() == 3:
        x = x[None]
    if not x.is_contiguous():
        raise ValueError("image must be contiguous")
    F, H, W, ch = x.shape
    if out is None:
        out = torch.empty((F, H, W), dtype=torch.float32, device=image.device)
    rc = lib.epic_gradient_cost(_ptr(x), F, H, W, ch, float(floor), _ptr(out),
                                _stream_handle(stream))
    if rc != EPIC_OK:
        raise EpicError(rc, "epic_gradient_cost")
    return out[0] if image.dim() < 4 else out
