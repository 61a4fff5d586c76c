"""Failure detection on the GPU without a fault: every device wait of the library is bounded.
A warp waits on a barrier phase that nothing completes, or on a completion counter that nothing
increments.  After the 2 s limit it records DWT2_ETIMEOUT in the workspace status word and
returns.  The host reads the status, and the context keeps working: a transform afterwards is
still exact."""
import time

import pytest
import torch

from paper_1708_07853_gb300 import dwt2 as D

pytestmark = pytest.mark.gpu

ETIMEOUT = 5


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1708_07853_gb300 import build as B
    B.build()


@pytest.mark.parametrize("which", [0, 1], ids=["barrier", "counter"])
def test_bounded_wait_reports_timeout_and_context_survives(which):
    ws = D.new_workspace(4096, "cuda")
    torch.cuda.synchronize()
    t0 = time.time()
    D.selftest_wait_timeout(which, ws)
    status = D.check_status(ws)  # synchronises
    elapsed = time.time() - t0
    assert status == ETIMEOUT
    assert 1.5 < elapsed < 60.0, elapsed
    x = torch.randint(-1000, 1000, (300, 517), dtype=torch.int32, device="cuda")
    c = D.forward(x, "cdf53_int", 3)
    assert torch.equal(D.inverse(c), x)
