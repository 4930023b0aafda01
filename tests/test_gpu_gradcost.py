"""Image-gradient cost map on the GPU (epic_gradient_cost) vs the oracle
(Table 2, "||grad_2 I||_2"): float32 arithmetic, so within 1e-6 relative +
1e-7 absolute of the FP64 value; frames of a stack are independent."""

import numpy as np
import pytest

import oracle
from paper_1501_02565_gb300 import synth
from parity import full_parity

pytestmark = pytest.mark.gpu


def _gpu(img, floor=0.0):
    import torch
    from paper_1501_02565_gb300.native import gradient_cost
    out = gradient_cost(torch.from_numpy(np.ascontiguousarray(img)).cuda(), floor)
    return out.cpu().numpy()


@pytest.mark.parametrize("shape", [(1, 1, 1), (1, 5, 3), (37, 70, 3), (64, 33, 4), (129, 257, 1)])
def test_random_images(shape):
    rng = np.random.default_rng(sum(shape))
    img = rng.uniform(0, 1, shape).astype(np.float32)
    g = _gpu(img, 1e-3)
    ref = oracle.gradient_cost(img, 1e-3)
    np.testing.assert_allclose(g, ref, rtol=1e-6, atol=1e-7)


def test_frame_stack_has_independent_borders():
    rng = np.random.default_rng(9)
    stack = rng.uniform(0, 1, (3, 20, 31, 3)).astype(np.float32)
    g = _gpu(stack)
    for f in range(3):
        np.testing.assert_allclose(g[f], oracle.gradient_cost(stack[f]), rtol=1e-6, atol=1e-7)


def test_gradient_cost_feeds_the_interpolator():
    # the cost of a synthetic region image drives the whole path, which
    # meets the usual parity rule
    p = synth.config_pair(1, 0)
    img = synth.region_image(p, seed=1)
    C = _gpu(img, 1e-3).astype(np.float32)
    np.testing.assert_allclose(C, oracle.gradient_cost(img, 1e-3), rtol=1e-6, atol=1e-7)
    assert C.max() < 2.0
    g, ref, rep = full_parity((C, p.matches), K=p.K, a=p.a)
    print("\n[gradcost] " + " ".join(f"{k}={v}" for k, v in rep.items()))
