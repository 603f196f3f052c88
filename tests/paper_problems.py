"""The fixed-point maps of the paper's experiments (Sec. 5), for tests.

Heat-2D with a nonlinear term (Sec. 5.1): u_xx + u_yy + c(u) = f on the
unit square, zero boundary, exact solution sin^2(pi x) sin^2(pi y), so
f = Lap(u_exact) + c(u_exact); discretised with second-order centred
differences, G(u) = A^{-1} (b - c(u)).  Bratu (Sec. 5.2):
u_xx + u_yy + lambda e^u = 0, G(u) = A^{-1} (-lambda e^u).

The paper solves with A by PCG and a multigrid preconditioner to 1e-10; here
A^{-1} is applied exactly through the type-I discrete sine transform, which
diagonalises the Dirichlet five-point Laplacian (scipy.fft.dstn).  Grid
index p = j*N + i with x_i = (i+1) h, h = 1/(N+1).
"""
from __future__ import annotations

import numpy as np
import scipy.fft as sf


class Poisson:
    def __init__(self, N: int):
        self.N = N
        h = 1.0 / (N + 1)
        k = np.arange(1, N + 1)
        lam1 = (2.0 * np.cos(np.pi * k * h) - 2.0) / h ** 2
        self.L = lam1[None, :] + lam1[:, None]
        x = np.arange(1, N + 1) * h
        self.X, self.Y = np.meshgrid(x, x, indexing="xy")

    def solve(self, r):
        R = np.asarray(r).reshape(self.N, self.N)
        return sf.idstn(sf.dstn(R, type=1) / self.L, type=1).reshape(-1)


def heat(N: int, term: int):
    """(G, u_exact) for Heat-2D with nonlinear term 1 or 2."""
    P = Poisson(N)
    X, Y = P.X, P.Y
    if term == 1:
        c = lambda u: u + u * np.exp(u) + u * np.exp(-u) + (u - np.exp(u)) ** 2
    else:
        c = lambda u: 100.0 * (u - u * u)
    ue = np.sin(np.pi * X) ** 2 * np.sin(np.pi * Y) ** 2
    pi2 = np.pi ** 2
    f = (2 * pi2 * (np.cos(np.pi * X) ** 2 - np.sin(np.pi * X) ** 2) * np.sin(np.pi * Y) ** 2
         + 2 * pi2 * (np.cos(np.pi * Y) ** 2 - np.sin(np.pi * Y) ** 2) * np.sin(np.pi * X) ** 2
         + c(ue)).reshape(-1)
    return (lambda u: P.solve(f - c(u))), ue.reshape(-1)


def bratu(N: int, lam: float):
    P = Poisson(N)
    return lambda u: P.solve(-lam * np.exp(u))


def em_mixture(copies: int, seed: int = 0, count: int = 100_000,
               alpha=(0.3, 0.3, 0.4), sigma=(1.0, 1.0, 1.0)):
    """The mixture-means EM map (Sec. 5.3): count samples from the poorly
    separated mixture with means (0, 0.5, 1) (aa_synth.mixture_samples), known
    proportions alpha and deviations sigma; one EM step replaces each mean by
    the posterior-weighted sample mean.  The three means are repeated copies
    times along the vector, as the paper does; every copy stays identical
    under AA (gamma is global), so G evaluates the first copy and repeats it.
    """
    import aa_synth
    X = aa_synth.mixture_samples(seed, count)
    al = np.asarray(alpha, dtype=np.float64)
    sg = np.asarray(sigma, dtype=np.float64)

    def step(mu):
        dens = al * np.exp(-(X[:, None] - mu[None, :]) ** 2 / (2.0 * sg ** 2)) / (np.sqrt(2.0 * np.pi) * sg)
        post = dens / dens.sum(axis=1, keepdims=True)
        return (post * X[:, None]).sum(axis=0) / post.sum(axis=0)

    def G(u):
        return np.tile(step(np.asarray(u[:3])), copies)

    return G, step
