"""Host model of the warp-tile relaxation's phase-2 work queue (no GPU).

The kernel's phase 2 hands out tiles through a queue without grid barriers:
a sweep over every tile, then the tiles a changed neighbour asked for.  Its
correctness rests on a small protocol: a per-tile state word (requested /
running / idle), a ring of pushed tiles read by tickets, and a busy count of
items not yet finished that tells a waiting warp when no item can come.

This model runs that protocol with simulated warps as generators that yield
at every step that touches shared state, under random interleavings.  The
"solve" of a tile is a relaxation step on a small grid graph: the tile's value
becomes the minimum of its own value and each neighbour's value plus an edge
weight, read one neighbour at a time (so other warps can write in between).
The model checks what the kernel relies on:

  * every schedule terminates (every warp leaves);
  * no tile is solved by two warps at once;
  * the values reach the fixed point that sequential Bellman-Ford reaches.
"""

import random

import numpy as np
import pytest

REQUESTED, RUNNING = 1, 2


class Shared:
    def __init__(self, values, weights, nbrs, chunk):
        self.v = list(values)
        self.w = weights
        self.nbrs = nbrs
        self.T = len(values)
        self.chunk = chunk
        self.n0 = (self.T + chunk - 1) // chunk
        self.head = 0
        self.tail = 0
        self.busy = self.T                    # the sweep's items
        self.state = [REQUESTED] * self.T     # every tile waits for the sweep
        self.ring = [-1] * self.T
        self.solving = [0] * self.T


def push(sh, t):
    """Ask for a solve of tile t (the kernel's queue_push)."""
    old = sh.state[t]
    sh.state[t] = old | REQUESTED
    yield
    if old != 0:
        return                                # queued already, or its warp solves it again
    sh.busy += 1
    yield
    p = sh.tail
    sh.tail += 1
    yield
    while sh.ring[p % sh.T] >= 0:             # the slot's previous item not taken yet
        yield
    sh.ring[p % sh.T] = t
    yield


def solve_item(sh, t):
    """One queue item (the kernel's solve_item)."""
    while True:
        sh.state[t] = RUNNING
        assert sh.solving[t] == 0, "tile solved by two warps at once"
        sh.solving[t] = 1
        yield
        best = sh.v[t]
        for n in sh.nbrs[t]:                  # neighbours read one at a time
            best = min(best, sh.v[n] + sh.w[(t, n)])
            yield
        changed = best < sh.v[t]
        if changed:
            sh.v[t] = best
            yield
        sh.solving[t] = 0
        if changed:
            for n in sh.nbrs[t]:
                yield from push(sh, n)
        old = sh.state[t]                     # compare-and-swap RUNNING -> idle
        if old == RUNNING:
            sh.state[t] = 0
        yield
        if old == RUNNING:
            break
    sh.busy -= 1
    yield


def warp(sh, solve):
    while True:
        h = sh.head
        sh.head += 1
        yield
        if h < sh.n0:
            for q in range(sh.chunk):
                t = h * sh.chunk + q
                if t < sh.T:
                    yield from solve(sh, t)
            continue
        p = h - sh.n0                         # the push this ticket takes
        while True:
            if sh.tail > p:
                while sh.ring[p % sh.T] < 0:
                    yield
                t = sh.ring[p % sh.T]
                sh.ring[p % sh.T] = -1
                yield
                yield from solve(sh, t)
                break
            if sh.busy == 0 and sh.tail <= p:
                return                        # no item will come
            yield
        continue


def fixed_point(values, weights, nbrs):
    v = list(values)
    while True:
        changed = False
        for t in range(len(v)):
            for n in nbrs[t]:
                if v[n] + weights[(t, n)] < v[t]:
                    v[t] = v[n] + weights[(t, n)]
                    changed = True
        if not changed:
            return v


def grid_case(rng, gw, gh):
    T = gw * gh
    nbrs = []
    weights = {}
    for t in range(T):
        x, y = t % gw, t // gw
        ns = []
        for dy in (-1, 0, 1):
            for dx in (-1, 0, 1):
                if (dx or dy) and 0 <= x + dx < gw and 0 <= y + dy < gh:
                    ns.append((y + dy) * gw + x + dx)
        nbrs.append(ns)
    for t in range(T):
        for n in nbrs[t]:
            if (n, t) in weights:
                weights[(t, n)] = weights[(n, t)]
            else:
                weights[(t, n)] = int(rng.integers(1, 20))
    big = 10 ** 6
    values = [int(rng.integers(0, 50)) if rng.random() < 0.15 else big for _ in range(T)]
    return values, weights, nbrs


@pytest.mark.parametrize("seed", range(40))
def test_random_schedules_terminate_at_the_fixed_point(seed):
    rng = np.random.default_rng(seed)
    gw, gh = int(rng.integers(2, 7)), int(rng.integers(2, 6))
    values, weights, nbrs = grid_case(rng, gw, gh)
    chunk = int(rng.integers(1, 5))
    sh = Shared(values, weights, nbrs, chunk)
    warps = [warp(sh, solve_item) for _ in range(int(rng.integers(1, 9)))]
    pick = random.Random(seed)
    live = list(warps)
    for _ in range(2_000_000):
        if not live:
            break
        g = pick.choice(live)
        try:
            next(g)
        except StopIteration:
            live.remove(g)
    assert not live, "a warp never left"
    assert sh.busy == 0
    assert sh.v == fixed_point(values, weights, nbrs)
    assert all(s == 0 for s in sh.state)


def solve_without_state(sh, t):
    """The protocol without the running state: a tile is idle as soon as it
    is taken, so a request during its solve pushes it again and another warp
    may solve it at the same time."""
    sh.state[t] = 0
    if sh.solving[t]:
        raise AssertionError("tile solved by two warps at once")
    sh.solving[t] = 1
    yield
    best = sh.v[t]
    for n in sh.nbrs[t]:
        best = min(best, sh.v[n] + sh.w[(t, n)])
        yield
    changed = best < sh.v[t]
    if changed:
        sh.v[t] = best
        yield
    sh.solving[t] = 0
    if changed:
        for n in sh.nbrs[t]:
            yield from push(sh, n)
    sh.busy -= 1
    yield


def test_the_model_sees_concurrent_solves():
    # without the running state some schedule solves a tile in two warps at
    # once; the model must see that, or the first test checks nothing
    seen = False
    for seed in range(200):
        rng = np.random.default_rng(seed)
        values, weights, nbrs = grid_case(rng, 4, 3)
        sh = Shared(values, weights, nbrs, 1)
        live = [warp(sh, solve_without_state) for _ in range(6)]
        pick = random.Random(seed)
        try:
            for _ in range(200_000):
                if not live:
                    break
                g = pick.choice(live)
                try:
                    next(g)
                except StopIteration:
                    live.remove(g)
        except AssertionError:
            seen = True
            break
    assert seen
