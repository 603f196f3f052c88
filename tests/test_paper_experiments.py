"""The oracle on the paper's own experiments (Sec. 5), as soft pins.

The paper prints iteration counts (its figures are not available):
- Heat-2D + nonlinear term 1, 1024^2, m = 5: 11 iterations for all variants
  (Sec. 5.1.1);
- Heat-2D + nonlinear term 2, 1024^2, m = 10: 27-42 iterations depending on
  variant and process count, CGS-2 best (Sec. 5.1.2); pinned here against a
  backward-stable least-squares reference (see the comment above its tests);
- Bratu, lambda = 6.7, 1024^2, m = 30: fewer than 30 iterations for all
  variants (Sec. 5.2).
The paper's G applies A^{-1} by PCG to 1e-10; here A^{-1} is exact (DST-I),
and the stop rule is Algorithm 1's ||x_{i+1} - x_i||_2 < 1e-10.  The
iteration counts therefore agree within one, not exactly.
"""
import numpy as np
import pytest

from paper_problems import bratu, heat

N = 1024


def solve(ora, G, m, orth, **kw):
    O = ora.Oracle(N * N, m, orth, **kw)
    with np.errstate(over="ignore", invalid="ignore"):
        return O.solve({"kind": "callback", "fn": G}, np.zeros(N * N), max_iters=80, tol=1e-10,
                       scale=1.0, stop_kind=1)


def test_heat_term1_eleven_iterations(ora):
    G, ue = heat(N, 1)
    its = []
    for orth in ["mgs", "icwy", "cgs2", "dcgs2"]:
        r = solve(ora, G, 5, orth)
        assert r["status"] == ora.OK
        its.append(r["iters"])
        # converged to the discrete solution: second-order close to the exact one
        assert np.max(np.abs(r["x"] - ue)) < 1e-5
    assert len(set(its)) == 1, its          # the same count for every variant
    assert abs(its[0] - 11) <= 1, its       # the paper: 11


def test_bratu_fewer_than_30(ora):
    G = bratu(N, 6.7)
    for orth, kw in [("mgs", {}), ("icwy", {}), ("cgs2", {}), ("dcgs2", {"dcgs2_scaled": True})]:
        r = solve(ora, G, 30, orth, **kw)
        assert r["status"] == ora.OK and r["iters"] < 30, (orth, r["iters"])


# Heat-2D + nonlinear term 2 (Sec. 5.1.2), c(u) = 100 (u - u^2), m = 10: the
# paper reports 27-42 iterations depending on the variant AND on the process
# count, i.e. on the order of the reductions -- a sign that this run is
# sensitive to rounding.  G is not a contraction here (c'(u) = 100 (1 - 2u)
# against the Laplacian's smallest eigenvalue 2 pi^2: a few modes are
# amplified about 5x), and the history becomes ill-conditioned (kappa(F) >
# 1e7 from iteration ~30, 1e12 near the end).  With the exact inner solve used
# here, the reference behaviour is Anderson acceleration with a backward-
# stable least-squares solve of the full history (Householder QR, no
# updating), which converges in 44 iterations at 1024^2.  The QR-updating
# variants whose Q loses orthogonality (MGS, ICWY: O(eps kappa) per update,
# accumulated across the updates; DCGS-2: its delayed reorthogonalisation,
# which the paper calls unstable) produce a least-squares solution gamma with
# O(1) error once kappa passes ~1e7 and diverge; CGS-2 keeps Q orthogonal to
# O(eps) and tracks the stable reference.


def householder_aa(G, x0, m, iters, tol):
    """Algorithm 1 by definition with a backward-stable least-squares solve
    (Householder QR of the explicit difference matrix, no updating).
    Returns (iterations to ||x_{i+1} - x_i||_2 < tol, x, per-step data)."""
    import scipy.linalg as sl
    g0 = G(x0)
    gs, fs, x = [g0], [g0 - x0], g0
    steps = []
    for i in range(1, iters + 1):
        g = G(x)
        f = g - x
        gs.append(g)
        fs.append(f)
        mi = min(m, i)
        dF = np.column_stack([fs[k + 1] - fs[k] for k in range(i - mi, i)])
        dG = np.column_stack([gs[k + 1] - gs[k] for k in range(i - mi, i)])
        Q, R = np.linalg.qr(dF)
        gamma = sl.solve_triangular(R, Q.T @ f)
        steps.append((fs[i] - fs[i - 1], f, gamma, dF))
        xn = g - dG @ gamma
        if np.linalg.norm(xn - x) < tol:
            return i, xn, steps
        x = xn
    return None, x, steps


def test_heat_term2_stable_reference_converges_in_44():
    G, ue = heat(N, 2)
    its, x, _ = householder_aa(G, np.zeros(N * N), 10, 60, 1e-10)
    assert its is not None and abs(its - 44) <= 1, its
    assert np.max(np.abs(x - ue)) < 1e-5


def test_heat_term2_cgs2_tracks_stable_reference(ora):
    G, ue = heat(N, 2)
    r = solve(ora, G, 10, "cgs2")
    assert r["status"] == ora.OK and abs(r["iters"] - 44) <= 1, r["iters"]
    assert np.max(np.abs(r["x"] - ue)) < 1e-5


def test_heat_term2_gamma_on_a_shared_history(ora):
    """The mechanism, on one history: the stable run's Delta f columns are
    fed to each variant's QR update, and its least-squares solution is
    compared with the Householder one at the steps where kappa(F) >= 1e7.
    CGS-2 keeps ||I - Q^T Q|| at the rounding level and gamma to 1e-8; MGS
    and ICWY have lost orthogonality (> 1e-6) and err by more than 1e-4."""
    n = 256
    G, _ = heat(n, 2)
    _, _, steps = householder_aa(G, np.zeros(n * n), 10, 34, 0.0)
    worst = {}
    for orth in ["mgs", "icwy", "cgs2"]:
        O = ora.Oracle(n * n, 10, orth)
        err, loss = 0.0, 0.0
        for df, f, gamma, dF in steps:
            assert O.qradd(df) == ora.OK
            if np.linalg.cond(dF) >= 1e7:
                go = O.lsq(f)
                Q, _, _ = O.get_qr()
                err = max(err, np.linalg.norm(go - gamma) / np.linalg.norm(gamma))
                loss = max(loss, np.linalg.norm(np.eye(Q.shape[1]) - Q.T @ Q))
        worst[orth] = (err, loss)
    assert worst["cgs2"][0] < 1e-8 and worst["cgs2"][1] < 1e-12, worst
    for orth in ["mgs", "icwy"]:
        assert worst[orth][0] > 1e-4 and worst[orth][1] > 1e-6, worst


# EM for the means of a three-component normal mixture (Sec. 5.3): AA(3),
# tolerance 1e-8 on ||x_{i+1} - x_i||_2, 21 iterations for every variant in
# the paper (one sample draw, initial means not stated; here mu_0 = (-1, 0, 1)).
EM_MU0 = (-1.0, 0.0, 1.0)


def em_solve(ora, G, copies, orth, max_iters=200):
    O = ora.Oracle(3 * copies, 3, orth)
    return O.solve({"kind": "callback", "fn": G}, np.tile(EM_MU0, copies), max_iters=max_iters,
                   tol=1e-8, scale=1.0, stop_kind=1)


def test_em_same_count_for_every_variant_near_21(ora):
    from paper_problems import em_mixture
    med = []
    for seed in range(5):
        G, step = em_mixture(1000, seed)
        its = []
        for orth in ["mgs", "icwy", "cgs2", "dcgs2"]:
            r = em_solve(ora, G, 1000, orth)
            assert r["status"] == ora.OK, (seed, orth)
            its.append(r["iters"])
            mu = r["x"][:3]
            # a fixed point of the EM map, and the copies stayed identical
            assert np.max(np.abs(step(mu) - mu)) < 1e-8
            assert np.max(np.abs(r["x"].reshape(-1, 3) - mu)) == 0.0
        # the same count up to one (rounding at the stop threshold)
        assert max(its) - min(its) <= 1, (seed, its)
        med.append(min(its))
    assert abs(np.median(med) - 21) <= 4, med


def test_em_aa_beats_plain_em(ora):
    from paper_problems import em_mixture
    G, step = em_mixture(1, 0)
    r = em_solve(ora, G, 1, "mgs")
    mu, k = np.array(EM_MU0), 0
    while k < 5000:
        mn = step(mu)
        k += 1
        if np.linalg.norm(mn - mu) < 1e-8:
            break
        mu = mn
    # the poorly separated mixture makes plain EM crawl
    assert k > 20 * r["iters"], (k, r["iters"])
    assert np.max(np.abs(mn - r["x"][:3])) < 1e-6
