"""The oracle's timed build (the same C source compiled with -fopenmp) against
its reference build: with one thread every sum runs in the same order, so the
iterates are bit-identical; with several threads the dot products are summed
in fixed chunks (one per thread) combined in chunk order, so the result is
reproducible run to run and agrees with the sequential sums to rounding."""
import numpy as np
import pytest

import aa_synth


def run(ora, omp, threads, orth, iters=12):
    nx, ny, nz = 23, 19, 17
    n = nx * ny * nz
    b = aa_synth.jacobi3d_rhs(0, nx, ny, nz)
    if omp:
        ora.set_threads(threads)
    O = ora.Oracle(n, 5, orth, omp=omp)
    x = np.zeros(n)
    out = []
    for _ in range(iters):
        g = ora.g_jacobi3d(nx, ny, nz, 0.1, 0.01, 0.8, b, x, omp=omp)
        x, fn, st = O.step(x, g)
        assert st == ora.OK
        out.append(x.copy())
    return out


@pytest.mark.parametrize("orth", ["mgs", "icwy", "cgs2", "dcgs2"])
def test_omp_one_thread_bit_identical(ora, orth):
    ref = run(ora, False, 1, orth)
    got = run(ora, True, 1, orth)
    assert all(np.array_equal(a, b) for a, b in zip(ref, got))


@pytest.mark.parametrize("orth", ["icwy", "cgs2"])
def test_omp_threads_reproducible_and_close(ora, orth):
    ref = run(ora, False, 1, orth)
    a = run(ora, True, 4, orth)
    b = run(ora, True, 4, orth)
    assert all(np.array_equal(x, y) for x, y in zip(a, b))
    for x, y in zip(ref, a):
        assert np.linalg.norm(x - y) <= 1e-11 * np.linalg.norm(y)
    ora.set_threads(1)
