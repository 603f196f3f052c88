"""Failure detection on the GPU without a fault: the bounded device-side
wait that every streaming pass uses on its mbarriers runs out on a barrier
that nothing completes, the kernel records the timeout and returns, the host
reads AA_ETIMEOUT, and the context keeps working."""
import time

import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu


def test_bounded_wait_times_out_and_context_survives():
    import paper_2110_09667_gb300 as aa
    t0 = time.time()
    rc = aa.selftest_wait_timeout()
    dt = time.time() - t0
    assert rc == -6, rc          # AA_ETIMEOUT
    assert dt < 60, dt           # the limit is about a second
    # the context is still usable: an AA step runs and gives finite output
    n = 1000
    A = aa.Anderson(n, 3, "icwy")
    x = torch.zeros(n, dtype=torch.float64, device="cuda")
    g = torch.ones(n, dtype=torch.float64, device="cuda")
    xn = torch.empty_like(x)
    fn = A.step(x, g, xn)
    assert fn == pytest.approx(np.sqrt(n))
    assert torch.equal(xn, g)
