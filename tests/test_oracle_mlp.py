"""Pins for the MLP oracle: gradients against central finite differences
(FP64), GELU against closed forms, bf16 rounding against known values."""
import math

import numpy as np

import aa_synth
from oracle import mlp


def params_for(dims, seed):
    out = []
    for li in range(len(dims) - 1):
        W = aa_synth.normal(seed + li, dims[li + 1] * dims[li]).reshape(dims[li + 1], dims[li]) * 0.5
        b = aa_synth.uniform(seed + 10 + li, dims[li + 1]) * 0.1
        out.append((W, b))
    return out


# GELU(z) = z Phi(z) at points where Phi, the standard normal CDF, has
# well-known tabulated values: Phi(1) = 0.8413447460685429,
# Phi(2) = 0.9772498680518208, Phi(3) = 0.9986501019683699, Phi(-z) = 1 - Phi(z);
# the density phi(1) = e^(-1/2) / sqrt(2 pi) = 0.24197072451914337.
GELU_TABLE = [
    (1.0, 0.8413447460685429),
    (-1.0, -(1.0 - 0.8413447460685429)),
    (2.0, 2.0 * 0.9772498680518208),
    (-2.0, -2.0 * (1.0 - 0.9772498680518208)),
    (3.0, 3.0 * 0.9986501019683699),
    (-3.0, -3.0 * (1.0 - 0.9986501019683699)),
]


def test_gelu_tabulated_values():
    for z, ref in GELU_TABLE:
        got = mlp.gelu(np.array([z]))[0]
        assert abs(got - ref) <= 4e-16 * max(1.0, abs(ref)), (z, got, ref)
    # derivative Phi(z) + z phi(z): 0.5 at 0, Phi(1) + phi(1) at 1, Phi(-1) - phi(1) at -1
    assert mlp.gelu_grad(np.array([0.0]))[0] == 0.5
    assert abs(mlp.gelu_grad(np.array([1.0]))[0] - (0.8413447460685429 + 0.24197072451914337)) < 1e-15
    assert abs(mlp.gelu_grad(np.array([-1.0]))[0]
               - ((1.0 - 0.8413447460685429) - 0.24197072451914337)) < 1e-15


def test_gelu_closed_forms():
    assert mlp.gelu(np.array([0.0]))[0] == 0.0
    assert abs(mlp.gelu(np.array([1.0]))[0] - 0.5 * (1 + math.erf(1 / math.sqrt(2)))) < 1e-16
    z = np.linspace(-4, 4, 41)
    fd = (mlp.gelu(z + 1e-6) - mlp.gelu(z - 1e-6)) / 2e-6
    assert np.max(np.abs(fd - mlp.gelu_grad(z))) < 1e-8


def test_gradients_match_finite_differences():
    dims = [5, 7, 6, 4]
    P = params_for(dims, 3)
    X = aa_synth.normal(7, 9 * 5).reshape(9, 5)
    T = aa_synth.normal(8, 9 * 4).reshape(9, 4)
    loss, _, grads = mlp.loss_and_grads(P, X, T)
    eps = 1e-6
    for li, (W, b) in enumerate(P):
        for idx in [(0, 0), (min(2, W.shape[0] - 1), 1), (W.shape[0] - 1, W.shape[1] - 1)]:
            Wp = [(w.copy(), bb.copy()) for w, bb in P]
            Wp[li][0][idx] += eps
            lp = mlp.loss_and_grads(Wp, X, T)[0]
            Wp[li][0][idx] -= 2 * eps
            lm = mlp.loss_and_grads(Wp, X, T)[0]
            assert abs((lp - lm) / (2 * eps) - grads[li][0][idx]) < 1e-7
        Bp = [(w.copy(), bb.copy()) for w, bb in P]
        Bp[li][1][0] += eps
        lp = mlp.loss_and_grads(Bp, X, T)[0]
        Bp[li][1][0] -= 2 * eps
        lm = mlp.loss_and_grads(Bp, X, T)[0]
        assert abs((lp - lm) / (2 * eps) - grads[li][1][0]) < 1e-7


def test_round_bf16():
    assert mlp.round_bf16(1.0) == 1.0
    assert mlp.round_bf16(1.0 + 2 ** -8) == 1.0  # tie to even
    assert mlp.round_bf16(1.0 + 3 * 2 ** -9) == 1.0 + 2 ** -7
    x = aa_synth.normal(1, 1000)
    r = mlp.round_bf16(x)
    assert np.max(np.abs(r - x) / np.abs(x)) <= 2 ** -8
