"""epic_interp_request_bytes (no GPU): the arena bytes the library reports for
one pair equal the carve-up of its scratch arena, rebuilt here from the
layout the library documents: every region 256-byte aligned, in the order
keys u64 [P]; seed bins int [T+1], [T], [N]; tile stamps [T]; edge table u64
and u32 [cap] with cap = max(1024, pow2 >= 8N); degree, lightest edge,
second-lightest edge, its other end [N] each; CSR row offsets [N+1] and
16-byte adjacency entries [2 cap]; models 2 x float4 [N]; fallback flags [N];
K-NN lists idx/dist [N x Kc] and counts [N] (only when intermediates are
kept); info int [4]; pruning buffers keep [N], float4 [N], int [N] (only when
pruning); plus one int per match in the batch's K-NN retry list and two ints
per relaxation tile (the relaxation's work queue and its queued flags)."""

import pytest

from paper_1501_02565_gb300 import native


def _a(x):
    return (x + 255) // 256 * 256


def carve(H, W, N, K, tile=(64, 16), keep=False, prune=False, prune_K=25):
    # the default configuration relaxes on warp tiles of 64 x 16
    P = H * W
    T = -(-W // tile[0]) * -(-H // tile[1])
    cap = 1024
    while cap < 8 * N:
        cap *= 2
    Kc = max(min(prune_K, N), min(K, N)) if prune else min(K, N)
    regions = [8 * P, 4 * (T + 1), 4 * T, 4 * N, 4 * T, 8 * cap, 4 * cap,
               4 * N, 4 * N, 4 * N, 4 * N, 4 * (N + 1), 16 * 2 * cap, 32 * N, 4 * N]
    if keep:
        regions += [4 * N * Kc, 4 * N * Kc, 4 * N]
    regions += [16]
    if prune:
        regions += [4 * N, 16 * N, 4 * N]
    return sum(_a(r) for r in regions) + 4 * N + 8 * T


@pytest.mark.parametrize("H, W, N, K", [(436, 1024, 5000, 100), (375, 1242, 8000, 100),
                                        (128, 256, 500, 32), (1, 1, 1, 1),
                                        (1080, 1920, 20000, 128), (37, 70, 30, 2048)])
@pytest.mark.parametrize("keep, prune", [(0, 0), (1, 0), (0, 1), (1, 1)])
def test_reported_bytes_equal_the_arena_carve_up(H, W, N, K, keep, prune):
    cfg = native.epic_config_default()
    cfg.keep_intermediates = keep
    cfg.prune = prune
    got = native.request_bytes(H, W, N, K, cfg=cfg)
    assert got == carve(H, W, N, K, keep=bool(keep), prune=bool(prune))


def test_refuses_sizes_a_run_would_refuse():
    for H, W, N, K in [(0, 5, 3, 3), (5, 5, 0, 3), (5, 5, 3, 0), (1 << 16, 1 << 15, 3, 3)]:
        with pytest.raises(native.EpicError):
            native.request_bytes(H, W, N, K)
