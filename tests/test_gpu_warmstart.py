"""Learned warm start, end to end at a small size (32 x 32 Bratu with
source): data from the batched solver, MLP trained with the library's
kernels, prediction used as x_0.  The trained network must cut the training
loss by 10x and reduce the mean iteration count of held-out solves versus
x_0 = 0 (every held-out solve still converging to 1e-8)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu


def test_warm_start_reduces_iterations():
    from paper_2110_09667_gb300 import warmstart as ws
    s = 32
    lam_tr, c_tr, src_tr = ws.instances(range(0, 384), s)
    U, it_tr, st_tr, _, _ = ws.solve_batch(lam_tr, src_tr, s, max_iters=20000)
    ok = st_tr == 0
    assert ok.mean() > 0.9
    X = ws.features(lam_tr[ok], c_tr[ok])
    net = ws.MLP(s * s, hidden=256, seed=1)
    hist = ws.train(net, X, U[ok], epochs=80, batch=64, lr=2e-3)
    assert hist[-1] < 0.1 * hist[0], hist[::10]
    lam_te, c_te, src_te = ws.instances(range(10000, 10064), s)
    _, it_cold, st_cold, _, _ = ws.solve_batch(lam_te, src_te, s, max_iters=20000)
    x0 = ws.predict(net, ws.features(lam_te, c_te))
    _, it_warm, st_warm, _, fb = ws.solve_batch(lam_te, src_te, s, x0=x0, max_iters=20000)
    good = st_cold == 0
    assert np.all(st_warm[good] == 0)
    assert fb.mean() < 0.5, fb
    assert it_warm[good].mean() < it_cold[good].mean(), (it_warm.mean(), it_cold.mean())
