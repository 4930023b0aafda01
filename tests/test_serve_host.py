"""Host-side request checks of the continuous-batching server (no GPU): a
request the device would reject is refused at submission, so it cannot fail a
batch it shares with other requests."""

import numpy as np
import pytest

from paper_1501_02565_gb300.native import EPIC_MAX_K
from paper_1501_02565_gb300.serve import Request, Server


def _request(N, K, H=60, W=80, a=1.0):
    rng = np.random.default_rng(N)
    C = rng.uniform(0.01, 1.0, (H, W)).astype(np.float32)
    flat = rng.choice(H * W, N, replace=False)
    m = np.zeros((N, 4), np.float32)
    m[:, 0], m[:, 1] = flat % W, flat // W
    m[:, 2:] = m[:, :2] + 1.5
    return Request(C, m, K, a)


def test_valid_requests_pass():
    Server.validate(_request(50, 10))
    # K above N is clamped to N, so only min(K, N) counts against the limit
    Server.validate(_request(50, 10 * EPIC_MAX_K))
    Server.validate(_request(EPIC_MAX_K, EPIC_MAX_K, H=64, W=64))


def test_k_above_the_search_table_limit_is_refused():
    with pytest.raises(ValueError, match="at most"):
        Server.validate(_request(EPIC_MAX_K + 1, EPIC_MAX_K + 1, H=64, W=64))


@pytest.mark.parametrize("K,a", [(0, 1.0), (5, 0.0), (5, -1.0), (5, float("nan"))])
def test_bad_k_or_a_is_refused(K, a):
    with pytest.raises(ValueError):
        Server.validate(_request(20, K, a=a))


def test_source_pixel_rounding_at_the_frame_edge():
    r = _request(5, 3, H=10, W=10)
    r.matches[0, :2] = (9.49, 9.49)       # rounds to pixel (9, 9): inside
    Server.validate(r)
    r.matches[0, :2] = (9.5, 0.0)         # rounds to column 10: outside
    with pytest.raises(ValueError, match="outside"):
        Server.validate(r)
    r.matches[0, :2] = (-0.51, 0.0)       # rounds to column -1: outside
    with pytest.raises(ValueError, match="outside"):
        Server.validate(r)


def test_non_finite_or_negative_cost_is_refused():
    r = _request(5, 3)
    r.C[2, 3] = -1e-3
    with pytest.raises(ValueError, match="cost"):
        Server.validate(r)
    r.C[2, 3] = np.inf
    with pytest.raises(ValueError, match="cost"):
        Server.validate(r)
