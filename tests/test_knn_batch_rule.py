"""The batched settle rule of the GPU K-NN search (stage c) reaches exactly
the neighbour lists of sequential Dijkstra under the key (distance, index)
(Algorithm 1 step 5), including ties and zero-weight edges.

The GPU search settles, in one step, every frontier node whose tentative
distance t is below B = min over the frontier of t(v) + w_x(v), where w_x(v)
is the lightest edge at v other than the edge to the settled node that gave
v its distance (the source uses its lightest edge), plus the smallest key.
A batch that would pass K is sorted by key and cut at K; one of more than 32
entries settles only its smallest key.  This is a host model of that rule,
compared with the oracle's Dijkstra on random graphs (no GPU)."""

import numpy as np
import pytest

import oracle


def batched_knn(adj, src, K, lane_cut=32, steps=None):
    """First K settled (distance, node) pairs under the batch rule; appends
    the number of steps taken to `steps` if given."""
    def w_x(v, parent):
        return min((w for x, w in adj[v] if x != parent), default=np.inf)

    t = {src: 0.0}
    settled = set()
    front = {src: (0.0, w_x(src, None))}      # node -> (t, t + w_x)
    out = []
    k = 0
    while len(out) < K and front:
        k += 1
        kmin = min((tv, v) for v, (tv, _) in front.items())
        bound = min(b for _, b in front.values())
        batch = sorted((tv, v) for v, (tv, _) in front.items() if tv < bound or (tv, v) == kmin)
        if len(out) + len(batch) >= K:
            if len(batch) <= lane_cut:
                out += batch[:K - len(out)]
                break
            batch = [kmin]
        for _, v in batch:
            settled.add(v)
            del front[v]
        out += batch
        for tv, v in batch:
            for u, w in adj[v]:
                nd = tv + w
                if u not in settled and (u not in t or nd < t[u]):
                    t[u] = nd
                    front[u] = (nd, nd + w_x(u, v))
    if steps is not None:
        steps.append(k)
    return out


def random_graph(rng, N, deg, wmax, zero_frac):
    """Connected graph: a random tree plus random extra edges; integer
    weights in [1, wmax] (many exact ties), a fraction of them zero."""
    edges = {(int(rng.integers(0, i)), i) for i in range(1, N)}
    target = min(N * deg // 2, N * (N - 1) // 2)
    while len(edges) < target:
        a, b = sorted(int(x) for x in rng.integers(0, N, 2))
        if a != b:
            edges.add((a, b))
    em, en = np.array(sorted(edges), np.int32).T.reshape(2, -1)
    ew = rng.integers(1, wmax + 1, len(em)).astype(np.float64)
    ew[rng.random(len(em)) < zero_frac] = 0.0
    adj = {i: [] for i in range(N)}
    for a, b, w in zip(em, en, ew):
        adj[int(a)].append((int(b), float(w)))
        adj[int(b)].append((int(a), float(w)))
    return adj, em, en, ew


@pytest.mark.parametrize("zero_frac", [0.0, 0.1])
@pytest.mark.parametrize("lane_cut", [32, 2])
def test_batched_rule_equals_dijkstra(zero_frac, lane_cut):
    rng = np.random.default_rng(17 + int(100 * zero_frac) + lane_cut)
    cases = 0
    for _ in range(60):
        N = int(rng.integers(2, 70))
        adj, em, en, ew = random_graph(rng, N, int(rng.integers(2, 9)),
                                       int(rng.integers(1, 5)), zero_frac)
        K = int(rng.integers(1, N + 1))
        idx, dist, cnt = oracle.knn(N, em, en, ew, K)
        for s in range(N):
            got = batched_knn(adj, s, K, lane_cut)
            assert len(got) == cnt[s]
            assert [v for _, v in got] == list(idx[s, :cnt[s]]), (N, K, s)
            np.testing.assert_array_equal([d for d, _ in got], dist[s, :cnt[s]])
            cases += 1
    assert cases > 500


def test_batches_settle_several_nodes_per_step():
    # the point of the rule: on a planar-like graph of positive weights a step
    # settles several nodes, so a search needs far fewer steps than K
    rng = np.random.default_rng(3)
    n = 30
    adj = {i: [] for i in range(n * n)}
    for y in range(n):
        for x in range(n):
            for dx, dy in ((1, 0), (0, 1)):
                if x + dx < n and y + dy < n:
                    w = float(rng.uniform(1.0, 1.2))
                    a, b = y * n + x, (y + dy) * n + x + dx
                    adj[a].append((b, w))
                    adj[b].append((a, w))
    K = 100
    steps = []
    for src in rng.choice(n * n, 20, replace=False):
        assert len(batched_knn(adj, int(src), K, steps=steps)) == K
    assert np.mean(steps) < K / 3
