"""Request dispatch over several GPUs: one continuous-batching server per
device, no collective on the data path (frame pairs are independent).

`Dispatcher` sends each request to the server with the least device memory
committed (admitted plus waiting requests, in bytes as the library sizes
them), ties to the server with the fewest waiting requests, then the lowest
device index, so large and small requests spread by the memory they hold
rather than by count.  Under torchrun, where every rank drives one GPU,
`rank_share` gives each rank its disjoint part of a request stream.
"""

from __future__ import annotations


class Dispatcher:
    """Least-loaded assignment of requests to per-device servers.  A server
    needs submit(req), load() -> committed bytes, a `pending` queue and
    stop(); serve.Server provides them."""

    def __init__(self, servers):
        if not servers:
            raise ValueError("need at least one server")
        self.servers = list(servers)
        self.assigned = [0] * len(self.servers)

    @classmethod
    def on_devices(cls, devices, **server_kw):
        """One started serve.Server per CUDA device index in `devices`."""
        from .serve import Server
        return cls([Server(d, **server_kw).start() for d in devices])

    def pick(self) -> int:
        best, best_key = 0, None
        for i, s in enumerate(self.servers):
            key = (s.load(), len(s.pending), i)
            if best_key is None or key < best_key:
                best, best_key = i, key
        return best

    def submit(self, req, **kw):
        """Submit `req` to the least-loaded server; returns (request, server
        index)."""
        i = self.pick()
        self.servers[i].submit(req, **kw)
        self.assigned[i] += 1
        return req, i

    def stop(self):
        """Drain and stop every server; the device status of each."""
        return [s.stop() for s in self.servers]

    def stats(self):
        """Per-server statistics and the request count each was given."""
        return [{"device_index": i, "assigned": n, **(s.stats() or {})}
                for i, (s, n) in enumerate(zip(self.servers, self.assigned))]


def rank_share(n_requests: int, rank: int, world: int):
    """Indices of a stream of n_requests that rank `rank` of `world` serves:
    request i goes to rank i mod world (arrival order interleaves the ranks,
    so each sees the same arrival rate)."""
    if not 0 <= rank < world:
        raise ValueError("rank out of range")
    return list(range(rank, n_requests, world))
