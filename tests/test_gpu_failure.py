"""Failure detection without a GPU fault: every device wait of the library
is bounded in time and reports EPIC_ERR_TIMEOUT; after such a report the
handle and the CUDA context stay usable."""

import numpy as np
import pytest

from paper_1501_02565_gb300 import synth

pytestmark = pytest.mark.gpu

EPIC_OK, EPIC_ERR_TIMEOUT = 0, 5


@pytest.mark.parametrize("which", [0, 1])   # grid barrier, TMA mbarrier
def test_bounded_wait_reports_timeout_and_context_survives(which):
    import time
    import torch
    from paper_1501_02565_gb300.native import EpicInterp
    p = synth.config_pair(1, 0)
    C = torch.from_numpy(p.C).cuda()
    M = torch.from_numpy(p.matches).cuda()
    eng = EpicInterp(0)
    ref = eng.run(C, M, p.K, p.a)
    eng.sync()
    ref = ref.cpu().numpy()
    t0 = time.monotonic()
    status = eng.selftest_wait_timeout(which, 50)
    took = time.monotonic() - t0
    assert status == EPIC_ERR_TIMEOUT
    assert took < 5.0
    # the same handle runs again and reproduces the result
    again = eng.run(C, M, p.K, p.a)
    assert eng.sync_status() == EPIC_OK
    assert np.array_equal(again.cpu().numpy(), ref)
    eng.close()
