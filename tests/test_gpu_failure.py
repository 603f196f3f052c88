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


def test_device_error_requires_reset_then_matches_oracle(ora):
    """A device-reported error leaves the history undefined: the call that
    reads it returns the code, later calls return AA_ESTATE until aa_reset,
    and after the reset the iterates match the oracle started afresh from
    the same point.  The failure is planted on the host (the status word is
    written as a timed-out pass would write it); no device fault."""
    import aa_synth
    import paper_2110_09667_gb300 as aa
    nx = ny = 64
    n = nx * ny
    b = aa_synth.jacobi2d_rhs(0, nx, ny)
    G = lambda x: ora.g_jacobi2d(nx, ny, 0.01, b, x)
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    A = aa.Anderson(n, 5, "icwy")
    x = np.zeros(n)
    xg = dev(x)
    xn = torch.empty_like(xg)
    for _ in range(8):
        A.step(xg, dev(G(xg.cpu().numpy())), xn)
        xg, xn = xn, xg
    A.test_set_device_status(-6)                   # AA_ETIMEOUT, as a pass would post it
    with pytest.raises(aa.AAError) as e:
        A.step(xg, dev(G(xg.cpu().numpy())), xn)
    assert e.value.code == -6
    with pytest.raises(aa.AAError) as e:           # refused until aa_reset
        A.step(xg, dev(G(xg.cpu().numpy())), xn)
    assert e.value.code == -8                      # AA_ESTATE
    with pytest.raises(aa.AAError) as e:
        A.qradd(xg)
    assert e.value.code == -8
    A.reset()
    O = ora.Oracle(n, 5, "icwy")
    xo = xg.cpu().numpy().copy()
    for i in range(25):
        xo_n, fo, st = O.step(xo, G(xo))
        fg = A.step(xg, dev(G(xg.cpu().numpy())), xn)
        xg, xn = xn, xg
        xo = xo_n
        assert abs(fg - fo) <= 1e-10 * abs(fo), (i, fg, fo)
        assert np.linalg.norm(xg.cpu().numpy() - xo) <= 1e-10 * np.linalg.norm(xo), i
