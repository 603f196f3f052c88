"""The GPU path on the paper's own experiments (Sec. 5) at full size
(1024^2 unknowns): every iteration goes through aa_step on the device; G
(an exact DST Poisson solve, see paper_problems.py) is evaluated on the host.
The iteration counts must equal the oracle's within one, under Algorithm 1's
stop rule ||x_{i+1} - x_i||_2 < 1e-10."""
import numpy as np
import pytest

from paper_problems import bratu, heat

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

N = 1024


def gpu_solve(aa, G, m, orth, flags=0, max_iters=80):
    A = aa.Anderson(N * N, m, orth, flags=flags)
    x = np.zeros(N * N)
    xd = torch.zeros(N * N, dtype=torch.float64, device="cuda")
    xn = torch.empty_like(xd)
    for i in range(max_iters):
        g = torch.from_numpy(G(x)).cuda()
        A.step(xd, g, xn)
        xnew = xn.cpu().numpy()
        if np.linalg.norm(xnew - x) < 1e-10:
            return i + 1, xnew
        x = xnew
        xd, xn = xn, xd
    return max_iters, x


def ora_solve(ora, G, m, orth, **kw):
    O = ora.Oracle(N * N, m, orth, **kw)
    return O.solve({"kind": "callback", "fn": G}, np.zeros(N * N), max_iters=80, tol=1e-10,
                   scale=1.0, stop_kind=1)


@pytest.mark.parametrize("orth", ["mgs", "icwy", "cgs2", "dcgs2"])
def test_heat_term1(ora, orth):
    import paper_2110_09667_gb300 as aa
    G, ue = heat(N, 1)
    it_g, xg = gpu_solve(aa, G, 5, orth)
    r = ora_solve(ora, G, 5, orth)
    assert abs(it_g - r["iters"]) <= 1, (it_g, r["iters"])
    assert np.max(np.abs(xg - ue)) < 1e-5


@pytest.mark.parametrize("orth", ["mgs", "icwy", "cgs2", "dcgs2"])
def test_bratu_67(ora, orth):
    import paper_2110_09667_gb300 as aa
    G = bratu(N, 6.7)
    scaled = orth == "dcgs2"
    it_g, xg = gpu_solve(aa, G, 30, orth, flags=aa.FLAG_DCGS2_SCALED if scaled else 0)
    r = ora_solve(ora, G, 30, orth, dcgs2_scaled=scaled)
    assert r["status"] == ora.OK and it_g < 30, (it_g, r["iters"])
    assert abs(it_g - r["iters"]) <= 1, (it_g, r["iters"])


@pytest.mark.parametrize("orth", ["mgs", "icwy", "cgs2", "dcgs2"])
def test_em_mixture(ora, orth):
    """EM for the mixture means (Sec. 5.3) at the paper's local vector size
    1.5e6 (500,000 copies of the three means), AA(3), tol 1e-8."""
    import paper_2110_09667_gb300 as aa
    from paper_problems import em_mixture
    copies = 500_000
    n = 3 * copies
    G, step = em_mixture(copies, 0)
    mu0 = np.tile([-1.0, 0.0, 1.0], copies)
    A = aa.Anderson(n, 3, orth)
    x = mu0.copy()
    xd = torch.from_numpy(x).cuda()
    xn = torch.empty_like(xd)
    it_g = None
    for i in range(200):
        g = torch.from_numpy(G(x)).cuda()
        A.step(xd, g, xn)
        xnew = xn.cpu().numpy()
        if np.linalg.norm(xnew - x) < 1e-8:
            it_g, x = i + 1, xnew
            break
        x = xnew
        xd, xn = xn, xd
    O = ora.Oracle(n, 3, orth)
    r = O.solve({"kind": "callback", "fn": G}, mu0, max_iters=200, tol=1e-8, scale=1.0, stop_kind=1)
    assert it_g is not None and r["status"] == ora.OK
    assert abs(it_g - r["iters"]) <= 1, (it_g, r["iters"])
    assert np.max(np.abs(x[:3] - r["x"][:3])) < 1e-7
    # every copy holds the same means
    assert np.max(np.abs(x.reshape(-1, 3) - x[:3])) < 1e-12
