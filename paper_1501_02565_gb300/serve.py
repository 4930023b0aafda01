"""Continuous-batching request loop for the interpolator.

Requests (one frame pair each: cost map, matches, K, a) arrive at any time.
A loop thread on the host:

1. admits waiting requests while the bytes they hold on the device (inputs,
   outputs and their share of the library's scratch) fit in the HBM budget
   and a batch slot is free; the admitted request's inputs are copied to the
   device on a copy stream, overlapping whatever batch is computing;
2. whenever the compute stream is idle, runs every admitted request whose
   upload has finished as ONE batched launch sequence
   (``epic_interp_run_batch``); requests that arrived meanwhile join the
   next step;
3. copies each finished flow back on the copy stream and completes the
   request when its CUDA event fires, releasing its budget and slot.

Latency is arrival -> completion on the host's monotonic clock.  Results do
not depend on which requests share a batch: every kernel computes a pair
from its own inputs only, so a request's flow is bit-identical alone and in
any mix.
"""

from __future__ import annotations

import collections
import dataclasses
import threading
import time

import numpy as np

from .native import EPIC_MAX_K, EpicInterp, request_bytes


@dataclasses.dataclass(eq=False)     # requests compare by identity
class Request:
    C: np.ndarray              # float32 [H, W]
    matches: np.ndarray        # float32 [N, 4]
    K: int
    a: float
    rid: int = 0
    arrival: float = 0.0       # host monotonic seconds
    admitted: float = 0.0
    completed: float = 0.0
    flow: object = None        # pinned torch tensor [H, W, 2] once done
    out: object = None         # optional caller-owned pinned [H, W, 2] output
    error: str | None = None
    _bytes: int = 0            # device bytes, set by the server at submission
    _done: threading.Event = dataclasses.field(default_factory=threading.Event)

    @property
    def H(self):
        return self.C.shape[0]

    @property
    def W(self):
        return self.C.shape[1]

    @property
    def P(self):
        return self.C.shape[0] * self.C.shape[1]

    def device_bytes(self, engine=None):
        """Device bytes the request holds while admitted: its cost map,
        matches and flow, plus the library's scratch for the pair as the
        library computes it (epic_interp_request_bytes) for `engine`'s
        configuration, or for the default configuration."""
        N = int(self.matches.shape[0])
        scratch = (engine.request_bytes(self.H, self.W, N, self.K) if engine is not None
                   else request_bytes(self.H, self.W, N, self.K))
        return int(self.P * (4 + 8) + N * 16 + scratch)

    def wait(self, timeout=None):
        if not self._done.wait(timeout):
            raise TimeoutError(f"request {self.rid} not completed")
        if self.error:
            raise RuntimeError(self.error)
        return self.flow

    @property
    def latency(self):
        return self.completed - self.arrival


class Server:
    """Continuous-batching interpolation server on one GPU."""

    def __init__(self, device: int = 0, max_batch: int = 32,
                 hbm_budget: int | None = None, reserve_bytes: int = 2 << 30,
                 max_pixels_per_batch: int = 64 << 20, **engine_cfg):
        import torch
        self.torch = torch
        self.device = device
        torch.cuda.set_device(device)
        self.dev = torch.device("cuda", device)
        self.max_batch = max_batch
        self.max_pixels = max_pixels_per_batch
        if hbm_budget is None:
            free, _ = torch.cuda.mem_get_info(device)
            hbm_budget = max(free - reserve_bytes, 256 << 20)
        self.budget = int(hbm_budget)
        self.in_use = 0
        engine_cfg.setdefault("use_graphs", 1)
        self.engine = EpicInterp(device, max_pairs=max_batch, **engine_cfg)
        self.compute = torch.cuda.Stream(device)
        self.copy = torch.cuda.Stream(device)
        self.pending = collections.deque()     # arrived, not admitted
        self.uploading = []                    # admitted, copy in flight
        self.inflight = []                     # (requests, done event) per step
        self.lock = threading.Lock()
        self.wake = threading.Condition(self.lock)
        self.running = False
        self.thread = None
        self.steps = 0
        self.batch_sizes = []
        self.completed = []
        self.max_in_use = 0

    # ------------------------------------------------------------------
    def start(self):
        self.running = True
        self.thread = threading.Thread(target=self._loop, daemon=True)
        self.thread.start()
        return self

    def stop(self):
        """Drain, stop the loop and return the device status (0 = every
        batch ran within its limits)."""
        with self.lock:
            self.running = False
            self.wake.notify_all()
        if self.thread:
            self.thread.join()
        status = self.engine.sync_status() if self.steps else 0
        self.engine.close()
        return status

    def load(self) -> int:
        """Device bytes this server has committed: admitted requests plus the
        ones waiting for admission (what a dispatcher balances on)."""
        with self.lock:
            return self.in_use + sum(r._bytes for r in self.pending)

    @staticmethod
    def validate(req: Request):
        """Host-side checks of what the device would otherwise report
        asynchronously (a match outside the frame, a non-finite or negative
        cost), so that a bad request is refused at submission."""
        C, m = req.C, req.matches
        C = C.numpy() if hasattr(C, "numpy") else C
        m = m.numpy() if hasattr(m, "numpy") else m
        if C.ndim != 2 or m.ndim != 2 or m.shape[1] != 4 or m.shape[0] < 1:
            raise ValueError("C must be [H, W] and matches [N, 4] with N >= 1")
        # two reductions: a NaN makes both comparisons false, +inf the second
        lo, hi = C.min(), C.max()
        if not (lo >= 0 and hi < np.inf):
            raise ValueError("cost map must be finite and >= 0")
        x = np.floor(m[:, 0].astype(np.float64) + 0.5)
        y = np.floor(m[:, 1].astype(np.float64) + 0.5)
        if not ((x >= 0) & (x < C.shape[1]) & (y >= 0) & (y < C.shape[0])).all():
            raise ValueError("a match's source pixel lies outside the frame")
        if req.K < 1 or not req.a > 0:
            raise ValueError("need K >= 1 and a > 0")
        if min(req.K, m.shape[0]) > EPIC_MAX_K:
            raise ValueError(f"K (clamped to N) must be at most {EPIC_MAX_K}")

    def submit(self, req: Request, validate: bool = True) -> Request:
        """Queue a request.  validate=False skips the host checks, for inputs
        the caller has already passed through Server.validate."""
        if self.thread is not None and not self.thread.is_alive():
            raise RuntimeError("the server loop is not running")
        if validate:
            self.validate(req)
        req._bytes = req.device_bytes(self.engine)
        if req._bytes > self.budget:
            raise ValueError(f"request {req.rid} needs more device memory than the budget")
        req.arrival = time.monotonic() if req.arrival == 0.0 else req.arrival
        with self.lock:
            self.pending.append(req)
            self.wake.notify_all()
        return req

    # ------------------------------------------------------------------
    def _admit(self):
        torch = self.torch
        admitted = []
        with self.lock:
            while self.pending and len(self.uploading) + len(admitted) < self.max_batch:
                r = self.pending[0]
                need = r._bytes
                if self.in_use + need > self.budget:
                    break
                self.pending.popleft()
                self.in_use += need
                self.max_in_use = max(self.max_in_use, self.in_use)
                admitted.append(r)
        for r in admitted:
            r.admitted = time.monotonic()
            with torch.cuda.stream(self.copy):
                hc = self._pinned(r.C)
                hm = self._pinned(r.matches)
                r._dC = hc.to(self.dev, non_blocking=True)
                r._dM = hm.to(self.dev, non_blocking=True)
                r._dF = torch.empty((r.H, r.W, 2), dtype=torch.float32, device=self.dev)
                r._hF = r.out if r.out is not None else torch.empty(
                    (r.H, r.W, 2), dtype=torch.float32, pin_memory=True)
                r._hold = (hc, hm)
        if admitted:
            up = torch.cuda.Event()
            up.record(self.copy)
            for r in admitted:
                r._up = up
                self.uploading.append(r)

    def _pinned(self, x):
        """Page-locked host copy of x (a pinned torch tensor is used as is)."""
        torch = self.torch
        if isinstance(x, torch.Tensor):
            return x if x.is_pinned() else x.contiguous().pin_memory()
        return torch.from_numpy(np.ascontiguousarray(x, np.float32)).pin_memory()

    def _launch(self):
        """Run every uploaded request as one batch if the compute stream is idle."""
        torch = self.torch
        # at most one batch queued behind the one computing: the GPU never
        # idles between steps, and new arrivals still join the next batch
        if sum(1 for _, _, c in self.inflight if not c.query()) >= 2:
            return False
        ready = [r for r in self.uploading if r._up.query()]
        if not ready:
            return False
        batch, px = [], 0
        for r in ready:
            if batch and (len(batch) >= self.max_batch or px + r.P > self.max_pixels):
                break
            batch.append(r)
            px += r.P
        for r in batch:
            self.uploading.remove(r)
        self.compute.wait_stream(self.copy)
        self.engine.run_batch([(r._dC, r._dM, r.K, r.a, r._dF) for r in batch],
                              stream=self.compute)
        comp_done = torch.cuda.Event()
        comp_done.record(self.compute)
        self.copy.wait_event(comp_done)
        with torch.cuda.stream(self.copy):
            for r in batch:
                r._hF.copy_(r._dF, non_blocking=True)
        done = torch.cuda.Event()
        done.record(self.copy)
        self.inflight.append((batch, done, comp_done))
        self.steps += 1
        self.batch_sizes.append(len(batch))
        return True

    def _complete(self):
        still = []
        finished = []
        for batch, done, comp in self.inflight:
            if done.query():
                finished.append(batch)
            else:
                still.append((batch, done, comp))
        self.inflight = still
        if not finished:
            return False
        now = time.monotonic()
        with self.lock:
            for batch in finished:
                for r in batch:
                    r.completed = now
                    r.flow = r._hF
                    for k in ("_dC", "_dM", "_dF", "_hold"):
                        setattr(r, k, None)
                    self.in_use -= r._bytes
                    self.completed.append(r)
                    r._done.set()
        return True

    def _loop(self):
        try:
            self._loop_body()
        except BaseException as exc:   # fail every outstanding request, never hang them
            msg = f"server loop failed: {exc!r}"
            with self.lock:
                self.running = False
                waiting = list(self.pending) + list(self.uploading)
                waiting += [r for batch, _, _ in self.inflight for r in batch]
                self.pending.clear()
                self.uploading = []
                self.inflight = []
                for r in waiting:
                    r.error = msg
                    r._done.set()
            raise

    def _loop_body(self):
        self.torch.cuda.set_device(self.device)
        while True:
            with self.lock:
                if not self.running and not self.pending and not self.uploading \
                        and not self.inflight:
                    return
                if not self.pending and not self.uploading and not self.inflight:
                    self.wake.wait(timeout=0.01)
                    continue
            progressed = self._complete()
            self._admit()
            progressed |= self._launch()
            if not progressed:
                time.sleep(20e-6)

    # ------------------------------------------------------------------
    def stats(self):
        lat = np.array([r.latency for r in self.completed])
        px = sum(r.P for r in self.completed)
        if not len(lat):
            return {}
        t0 = min(r.arrival for r in self.completed)
        t1 = max(r.completed for r in self.completed)
        return {
            "requests": len(lat),
            "latency_ms_p50": float(np.percentile(lat, 50) * 1e3),
            "latency_ms_p99": float(np.percentile(lat, 99) * 1e3),
            "mpix_s": px / max(t1 - t0, 1e-9) / 1e6,
            "steps": self.steps,
            "mean_batch": float(np.mean(self.batch_sizes)) if self.batch_sizes else 0.0,
        }


def replay(server: Server, requests, arrivals, validate: bool = True):
    """Submit `requests` at the given offsets (seconds from now) and wait.
    A request's latency counts from its scheduled arrival, so a submitter
    that falls behind the schedule adds to the measured latency."""
    t0 = time.monotonic()
    for r, t in zip(requests, arrivals):
        delay = t0 + t - time.monotonic()
        if delay > 0:
            time.sleep(delay)
        r.arrival = t0 + t
        server.submit(r, validate=validate)
    for r in requests:
        r.wait(timeout=120)
    return server.stats()
