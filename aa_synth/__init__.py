"""Seeded synthetic inputs for the Anderson-acceleration workloads.

This module is the one piece shared by the CPU oracle's tests and the GPU
path's tests and benchmark. It holds random-number generation and problem
*parameters* only (right-hand sides, grid sizes, Bratu parameters, test
matrices), never any step of Anderson acceleration or of the QR updates.

Random numbers come from SplitMix64 (Steele, Lea and Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014) used as a counter-based
generator: value i of stream ``seed`` is ``mix(key(seed) + (i + 1) * GOLDEN)``.
Uniforms take the top 53 bits; normals use the Box-Muller transform on two
independent uniform streams.
"""
from __future__ import annotations

import math

import numpy as np

GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def _mix(z: np.ndarray) -> np.ndarray:
    """SplitMix64 output function (the published finaliser)."""
    z = z.copy()
    z ^= z >> np.uint64(30)
    z *= _M1
    z ^= z >> np.uint64(27)
    z *= _M2
    z ^= z >> np.uint64(31)
    return z


def _key(seed: int, stream: int) -> np.uint64:
    s = np.array([(seed * 1_000_003 + stream) & 0xFFFFFFFFFFFFFFFF], dtype=np.uint64)
    return _mix(s + GOLDEN)[0]


def u64(seed: int, n: int, stream: int = 0, offset: int = 0) -> np.ndarray:
    """n raw 64-bit outputs of stream (seed, stream), starting at counter offset."""
    with np.errstate(over="ignore"):
        i = np.arange(offset + 1, offset + n + 1, dtype=np.uint64)
        return _mix(_key(seed, stream) + i * GOLDEN)


def uniform(seed: int, n: int, lo: float = -1.0, hi: float = 1.0, stream: int = 0,
            chunk: int = 1 << 24) -> np.ndarray:
    """n doubles uniform on [lo, hi) from the top 53 bits of each output.

    Generated in chunks so that multi-GB vectors do not need multi-GB
    temporaries."""
    out = np.empty(n, dtype=np.float64)
    for s in range(0, n, chunk):
        e = min(n, s + chunk)
        r = u64(seed, e - s, stream, offset=s)
        u = (r >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)
        out[s:e] = lo + (hi - lo) * u
    return out


def normal(seed: int, n: int, stream: int = 0) -> np.ndarray:
    """n standard normals by Box-Muller on two uniform streams."""
    u1 = uniform(seed, n, 0.0, 1.0, stream=2 * stream + 101)
    u2 = uniform(seed, n, 0.0, 1.0, stream=2 * stream + 102)
    u1 = 1.0 - u1  # (0, 1]
    return np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * math.pi * u2)


# ---------------------------------------------------------------------------
# Workload parameters
# ---------------------------------------------------------------------------

def jacobi2d_rhs(seed: int, nx: int, ny: int) -> np.ndarray:
    """b ~ U(-1, 1) for the 2D anisotropic Jacobi problem (x fastest)."""
    return uniform(seed, nx * ny, stream=1)


def jacobi3d_rhs(seed: int, nx: int, ny: int, nz: int) -> np.ndarray:
    """b ~ U(-1, 1) for the 3D anisotropic weighted-Jacobi problem."""
    return uniform(seed, nx * ny * nz, stream=2)


def bratu_batch(seed: int, count: int, side_lo: int = 32, side_hi: int = 256,
                lam_lo: float = 1.0, lam_hi: float = 6.0):
    """Batched Bratu parameters: side ~ round(exp(U(ln lo, ln hi))), lambda ~ U(lo, hi)."""
    ul = uniform(seed, count, math.log(side_lo), math.log(side_hi), stream=3)
    sides = np.clip(np.rint(np.exp(ul)).astype(np.int64), side_lo, side_hi)
    lams = uniform(seed, count, lam_lo, lam_hi, stream=4)
    return sides, lams


def bratu_source_params(seed: int, modes: int = 8, lam_lo: float = 1.0, lam_hi: float = 6.0):
    """Parametric Bratu-with-source instance: (lambda, c) with c_k ~ N(0, 1),
    k over modes x modes sine modes (row-major in (k1, k2))."""
    lam = float(uniform(seed, 1, lam_lo, lam_hi, stream=5)[0])
    c = normal(seed, modes * modes, stream=6)
    return lam, c


def dense_contraction(seed: int, n: int, rho: float = 0.9):
    """A dense linear fixed-point map G(x) = M x + c with spectral norm rho.

    M = rho * U diag(d) V^T with U, V products of random Householder
    reflections and d in [0.1, 1]; c ~ U(-1, 1)."""
    U = householder_orthogonal(seed, n, n, stream=7)
    V = householder_orthogonal(seed, n, n, stream=8)
    d = uniform(seed, n, 0.1, 1.0, stream=9)
    d[0] = 1.0
    M = rho * (U * d) @ V.T
    c = uniform(seed, n, stream=10)
    return M, c


def householder_orthogonal(seed: int, n: int, k: int, stream: int = 11, reflections: int = 0):
    """First k columns of a random n x n orthogonal matrix, built as a product of
    Householder reflections I - 2 w w^T / (w^T w) with Gaussian w."""
    nref = reflections or min(n, k + 2)
    Qm = np.eye(n, k)
    for r in range(nref):
        w = normal(seed, n, stream=1000 * stream + r)
        Qm = Qm - np.outer(w, (2.0 / (w @ w)) * (w @ Qm))
    return Qm


def matrix_with_condition(seed: int, n: int, m: int, kappa: float) -> np.ndarray:
    """n x m matrix with singular values logspaced from 1 to 1/kappa."""
    U = householder_orthogonal(seed, n, m, stream=12)
    V = householder_orthogonal(seed, m, m, stream=13)
    s = np.logspace(0.0, -math.log10(kappa), m)
    return (U * s) @ V.T


def bratu_source_grid(c: np.ndarray, s: int, modes: int = 8) -> np.ndarray:
    """Source f on the s x s interior grid (x_i = i h, h = 1/(s+1), index
    p = j*s + i) for sine-mode coefficients c (modes x modes, row-major in
    (k1, k2)): f(x, y) = sum_{k1,k2} c[k1,k2] / (k1^2 + k2^2) sin(k1 pi x) sin(k2 pi y)."""
    k = np.arange(1, modes + 1)
    x = np.arange(1, s + 1) / (s + 1.0)
    S = np.sin(np.pi * np.outer(x, k))  # [s, modes]
    W = np.asarray(c, dtype=np.float64).reshape(modes, modes) / (k[:, None] ** 2 + k[None, :] ** 2)
    F = S @ W.T @ S.T  # F[j, i]: y index j, x index i
    return F.reshape(-1)


def mixture_samples(seed: int, count: int, alpha=(0.3, 0.3, 0.4), mu=(0.0, 0.5, 1.0),
                    sigma=(1.0, 1.0, 1.0)) -> np.ndarray:
    """count draws from the univariate normal mixture sum_i alpha_i N(mu_i, sigma_i^2):
    the component by inverting the cumulative proportions on a uniform, the value
    by a standard normal scaled and shifted."""
    u = uniform(seed, count, 0.0, 1.0, stream=7)
    z = normal(seed, count, stream=8)
    comp = np.searchsorted(np.cumsum(alpha)[:-1], u, side="right")
    return np.asarray(mu, dtype=np.float64)[comp] + np.asarray(sigma, dtype=np.float64)[comp] * z
