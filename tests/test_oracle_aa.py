"""Pins for the oracle's Anderson iteration (Algorithm 1 with Algorithm 2).

- brute-force AA written from the definition in Algorithm 1 (explicit
  difference histories, SVD least squares, no QR updating);
- the equivalence of untruncated AA and GMRES for linear maps (the paper's
  introduction, after Walker and Ni): x^{AA}_{k+1} = G(x^{GMRES}_k);
- the secant identity for n = 1 and finite termination for linear maps;
- the stencil maps against dense-matrix constructions.
"""
import numpy as np
import pytest

import aa_synth

VARIANTS = ["mgs", "icwy", "cgs2", "dcgs2"]


def aa_bruteforce(G, x0, m, iters):
    """Algorithm 1 by definition: gamma = argmin ||f_i - F_i gamma|| by SVD."""
    g0 = G(x0)
    xs, gs, fs = [x0], [g0], [g0 - x0]
    x = g0
    out = [x]
    for i in range(1, iters + 1):
        g = G(x)
        f = g - x
        xs.append(x)
        gs.append(g)
        fs.append(f)
        mi = min(m, i)
        dF = np.column_stack([fs[k + 1] - fs[k] for k in range(i - mi, i)])
        dG = np.column_stack([gs[k + 1] - gs[k] for k in range(i - mi, i)])
        gamma = np.linalg.lstsq(dF, f, rcond=None)[0]
        x = g - dG @ gamma
        out.append(x)
    return out


def aa_oracle(ora, G, x0, m, iters, orth, **kw):
    O = ora.Oracle(len(x0), m, orth, **kw)
    x = x0.copy()
    out = []
    for _ in range(iters + 1):
        xn, _, st = O.step(x, G(x))
        assert st == ora.OK
        out.append(xn)
        x = xn
    return out


@pytest.mark.parametrize("orth", VARIANTS)
@pytest.mark.parametrize("m", [1, 3, 6])
def test_aa_matches_definition(ora, orth, m):
    """Iterates of the QR-updating oracle equal brute-force AA (including
    the truncated regime where QRDelete runs)."""
    M, c = aa_synth.dense_contraction(20, 40, rho=0.95)
    G = lambda x: M @ x + c
    x0 = np.zeros(40)
    iters = 12
    ref = aa_bruteforce(G, x0, m, iters)
    got = aa_oracle(ora, G, x0, m, iters, orth)
    for i, (a, b) in enumerate(zip(got, ref)):
        assert np.linalg.norm(a - b) <= 1e-9 * np.linalg.norm(b), (i, orth, m)


def test_aa_matches_definition_nonlinear(ora):
    """Same on a nonlinear map (Bratu nonlinear Jacobi, 12 x 12)."""
    s, lam = 12, 3.0
    G = lambda u: ora.g_bratu2d(s, lam, None, u)
    x0 = np.zeros(s * s)
    ref = aa_bruteforce(G, x0, 4, 10)
    for orth in VARIANTS:
        got = aa_oracle(ora, G, x0, 4, 10, orth)
        for a, b in zip(got, ref):
            assert np.linalg.norm(a - b) <= 1e-9 * np.linalg.norm(b)


def gmres_bruteforce(A, bvec, x0, k):
    """x_k = argmin over x0 + K_k(A, r0) of ||b - A x|| (dense)."""
    r0 = bvec - A @ x0
    K = np.column_stack([np.linalg.matrix_power(A, j) @ r0 for j in range(k)])
    V, _ = np.linalg.qr(K)
    y = np.linalg.lstsq(A @ V, r0, rcond=None)[0]
    return x0 + V @ y


@pytest.mark.parametrize("orth", VARIANTS)
def test_aa_gmres_equivalence(ora, orth):
    n = 30
    M, c = aa_synth.dense_contraction(21, n, rho=0.9)
    G = lambda x: M @ x + c
    A = np.eye(n) - M
    x0 = aa_synth.uniform(22, n) * 0.1
    got = aa_oracle(ora, G, x0, 20, 8, orth)  # got[k] = x_{k+1}
    for k in range(1, 8):
        xg = gmres_bruteforce(A, c, x0, k)
        target = G(xg)
        assert np.linalg.norm(got[k] - target) <= 1e-8 * np.linalg.norm(target), (orth, k)


def test_secant_n1(ora):
    """n = 1, G(x) = a x + c: x_2 is the exact fixed point (secant step)."""
    a, c = 0.7, 1.3
    G = lambda x: a * x + c
    for orth in VARIANTS:
        got = aa_oracle(ora, G, np.array([0.25]), 1, 1, orth)
        assert abs(got[1][0] - c / (1 - a)) < 1e-14


def test_finite_termination(ora):
    """Linear G in R^n with m >= n: residual vanishes by iteration n + 1."""
    n = 6
    M, c = aa_synth.dense_contraction(23, n, rho=0.8)
    for orth in ["mgs", "icwy", "cgs2"]:
        O = ora.Oracle(n, 10, orth)
        x = np.zeros(n)
        f0 = None
        for i in range(n + 2):
            xn, fn, st = O.step(x, M @ x + c)
            f0 = fn if f0 is None else f0
            if st == ora.BREAKDOWN:  # the history spans R^n: done
                break
            x = xn
        assert np.linalg.norm(M @ x + c - x) < 1e-9 * f0


# ------------------------------------------------------------- problem maps

def lap1d(n):
    return 2 * np.eye(n) - np.eye(n, k=1) - np.eye(n, k=-1)


def test_jacobi2d_map_dense(ora):
    nx, ny, eps = 5, 4, 0.01
    A = np.kron(np.eye(ny), lap1d(nx)) + eps * np.kron(lap1d(ny), np.eye(nx))
    b = aa_synth.jacobi2d_rhs(0, nx, ny)
    x = aa_synth.uniform(1, nx * ny)
    d = np.diag(A)
    assert np.allclose(d, 2 + 2 * eps)
    ref = x + (b - A @ x) / d
    assert np.max(np.abs(ora.g_jacobi2d(nx, ny, eps, b, x) - ref)) < 1e-15
    # fixed point is the solution of A x = b
    xs = np.linalg.solve(A, b)
    assert np.max(np.abs(ora.g_jacobi2d(nx, ny, eps, b, xs) - xs)) < 1e-13


def test_jacobi3d_map_dense(ora):
    nx, ny, nz, ey, ez, om = 4, 3, 5, 0.1, 0.01, 0.8
    I = np.eye
    A = (np.kron(I(nz), np.kron(I(ny), lap1d(nx))) + ey * np.kron(I(nz), np.kron(lap1d(ny), I(nx)))
         + ez * np.kron(lap1d(nz), np.kron(I(ny), I(nx))))
    b = aa_synth.jacobi3d_rhs(0, nx, ny, nz)
    x = aa_synth.uniform(2, nx * ny * nz)
    assert np.allclose(np.diag(A), 2 * (1 + ey + ez))
    ref = x + om * (b - A @ x) / np.diag(A)
    assert np.max(np.abs(ora.g_jacobi3d(nx, ny, nz, ey, ez, om, b, x) - ref)) < 1e-15


def test_bratu_map_closed_form(ora):
    """Bratu nonlinear Jacobi: G(u) = (sum nbrs + h^2 (lam e^u + src)) / 4;
    at u = 0 it is h^2 (lam + src) / 4 everywhere; on a dense Laplacian its
    fixed point satisfies the discrete Bratu equation."""
    s, lam = 6, 2.0
    h2 = 1.0 / (s + 1) ** 2
    src = aa_synth.uniform(3, s * s)
    g0 = ora.g_bratu2d(s, lam, src, np.zeros(s * s))
    assert np.max(np.abs(g0 - h2 * (lam + src) / 4)) < 1e-16
    L = (np.kron(np.eye(s), lap1d(s)) + np.kron(lap1d(s), np.eye(s)))
    u = aa_synth.uniform(4, s * s) * 0.1
    ref = ((4 * np.eye(s * s) - L) @ u + h2 * (lam * np.exp(u) + src)) / 4
    assert np.max(np.abs(ora.g_bratu2d(s, lam, src, u) - ref)) < 1e-15


def test_solve_jacobi2d_small(ora):
    """The oracle's solve loop reaches the stated stop rule on the small
    2D problem (64 x 64 is exercised in the GPU parity tests)."""
    nx = ny = 16
    b = aa_synth.jacobi2d_rhs(0, nx, ny)
    O = ora.Oracle(nx * ny, 5, "mgs")
    r = O.solve({"kind": "jacobi2d", "nx": nx, "ny": ny, "eps": 0.01, "b": b},
                np.zeros(nx * ny), max_iters=500, tol=1e-8, scale=np.linalg.norm(b))
    assert r["status"] == ora.OK
    x = r["x"]
    res = np.linalg.norm(ora.g_jacobi2d(nx, ny, 0.01, b, x) - x) / np.linalg.norm(b)
    assert res < 1e-8
    assert r["resid"][-1] / np.linalg.norm(b) < 1e-8
    assert r["resid"][-2] / np.linalg.norm(b) >= 1e-8
