"""Warm-start MLP kernels against numpy / the FP64 MLP oracle.

GEMM: BF16 inputs are exact in FP64, products are exact in FP32, the FP32
accumulation over K terms errs by at most K * 2^-24 relative to
sum |a_i b_i|; the test allows 2 K 2^-24.  MLP gradients: activations and
gradients are rounded to BF16 between layers (2^-8 relative each), so the
GPU gradients are compared with the FP64 oracle by relative norm (5e-2) and
direction (cosine > 0.998).
"""
import numpy as np
import pytest

import aa_synth
from oracle import mlp as omlp

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ws():
    import paper_2110_09667_gb300 as aa
    from paper_2110_09667_gb300 import warmstart
    aa.lib()
    return warmstart


def bf16(a):
    return torch.from_numpy(omlp.round_bf16(a).astype(np.float32)).cuda().to(torch.bfloat16)


IMPLS = ["tc", "mma"]


def _tc_ok(ws, impl):
    if impl == "tc":
        ws.gemm_tc_status()  # raises on a timed-out tcgen05 CTA


@pytest.mark.parametrize("impl", IMPLS)
@pytest.mark.parametrize("M,N,K", [(200, 300, 136), (1, 8, 8), (129, 1, 64), (256, 1024, 72)])
def test_gemm_nt(ws, impl, M, N, K):
    A = omlp.round_bf16(aa_synth.normal(1, M * K).reshape(M, K))
    B = omlp.round_bf16(aa_synth.normal(2, N * K).reshape(N, K))
    C = torch.empty(M, N, dtype=torch.float32, device="cuda")
    ws.gemm_nt(bf16(A), bf16(B), C, impl=impl)
    _tc_ok(ws, impl)
    ref = A @ B.T
    bound = 2 * K * 2.0 ** -24 * (np.abs(A) @ np.abs(B).T)
    assert np.all(np.abs(C.cpu().numpy() - ref) <= bound + 1e-30)


# tcgen05 path: both tile widths (128 x 256 once the grid has >= 148 such
# tiles), many K blocks through the stage ring, ragged M, N and K, a leading
# dimension larger than the row, and the persistent form (more than two
# tiles per SM: 336 tiles of 128 x 256, 313 of 128 x 128)
@pytest.mark.parametrize("M,N,K,lda", [(1280, 4096, 136, 136), (300, 520, 1000, 1000),
                                       (130, 257, 8, 16), (128, 1024, 1024, 1032),
                                       (1300, 4000, 72, 72), (2577, 4056, 200, 200),
                                       (40003, 120, 64, 72)])
def test_gemm_tc_shapes(ws, M, N, K, lda):
    A = omlp.round_bf16(aa_synth.normal(41, M * K).reshape(M, K))
    B = omlp.round_bf16(aa_synth.normal(42, N * K).reshape(N, K))
    Ad = torch.zeros(M, lda, dtype=torch.bfloat16, device="cuda")
    Ad[:, :K] = bf16(A)
    C = torch.full((M, N), float("nan"), dtype=torch.float32, device="cuda")
    ws.gemm_nt(Ad[:, :K], bf16(B), C, impl="tc")
    ws.gemm_tc_status()
    ref = A @ B.T
    bound = 2 * K * 2.0 ** -24 * (np.abs(A) @ np.abs(B).T)
    c = C.cpu().numpy()
    assert np.all(np.isfinite(c))
    assert np.all(np.abs(c - ref) <= bound + 1e-30)
    # the two tensor-core paths compute the same sums up to their order
    C2 = torch.empty_like(C)
    ws.gemm_nt(Ad[:, :K], bf16(B), C2, impl="mma")
    assert np.all(np.abs(C2.cpu().numpy() - c) <= 2 * bound + 1e-30)


@pytest.mark.parametrize("impl", IMPLS)
def test_gemm_epilogue(ws, impl):
    M, N, K = 70, 90, 40
    A = omlp.round_bf16(aa_synth.normal(3, M * K).reshape(M, K))
    B = omlp.round_bf16(aa_synth.normal(4, N * K).reshape(N, K))
    bias = aa_synth.uniform(5, N).astype(np.float32)
    H = torch.empty(M, N, dtype=torch.bfloat16, device="cuda")
    P = torch.empty(M, N, dtype=torch.float32, device="cuda")
    ws.gemm_nt(bf16(A), bf16(B), H, bias=torch.from_numpy(bias).cuda(), pre=P,
               epi=ws.EPI_BIAS | ws.EPI_GELU | ws.EPI_BF16 | ws.EPI_PRE, impl=impl)
    _tc_ok(ws, impl)
    pre = A @ B.T + bias.astype(np.float64)
    assert np.max(np.abs(P.cpu().numpy() - pre)) < 1e-4 * np.abs(pre).max()
    h = H.float().cpu().numpy()
    assert np.max(np.abs(h - omlp.gelu(pre)) / (np.abs(omlp.gelu(pre)) + 1e-3)) < 2 ** -7


def test_transpose(ws):
    X = bf16(aa_synth.normal(6, 37 * 53).reshape(37, 53))
    out = torch.empty(53, 37, dtype=torch.bfloat16, device="cuda")
    ws.transpose(X, out)
    assert torch.equal(out, X.t().contiguous())


@pytest.mark.parametrize("impl", IMPLS)
def test_mlp_gradients_vs_oracle(ws, impl, monkeypatch):
    """Forward output and parameter gradients of the GPU MLP (kernels only)
    against the FP64 oracle MLP, on the same BF16 weights and inputs."""
    monkeypatch.setattr(ws, "GEMM_IMPL", impl)
    out_dim, hidden, Bn = 48, 64, 32
    net = ws.MLP(out_dim, hidden=hidden, seed=3)
    # the output layer starts at zero in training; give it random weights so
    # that every layer's gradient is nonzero here
    W3, Wb3, _ = net.params[2]
    W3.copy_(torch.from_numpy((aa_synth.normal(13, W3.numel()).reshape(W3.shape) / 8.0)
                              .astype(np.float32)).cuda())
    assert ws._L().aa_f32_to_bf16(W3.numel(), ws._p(W3), ws._p(Wb3), ws._stream()) == 0
    P = []
    for W, Wb, b in net.params:
        P.append((Wb.float().cpu().numpy().astype(np.float64), b.cpu().numpy().astype(np.float64)))
    X = np.zeros((Bn, ws.IN_PAD))
    X[:, :ws.IN_DIM] = omlp.round_bf16(aa_synth.normal(9, Bn * ws.IN_DIM).reshape(Bn, ws.IN_DIM))
    T = aa_synth.normal(10, Bn * out_dim).reshape(Bn, out_dim)
    Xd = bf16(X)
    Td = torch.from_numpy(T.astype(np.float32)).cuda()
    Y = net.forward(Xd)
    loss, dY = net.loss_and_grad(Y, Td)
    grads = net.backward(dY)
    torch.cuda.synchronize()
    oloss, oY, ograds = omlp.loss_and_grads(P, X, T)
    y = Y.cpu().numpy()
    assert np.linalg.norm(y - oY) <= 2e-2 * np.linalg.norm(oY)
    assert abs(loss - oloss) <= 2e-2 * oloss
    for li in range(3):
        for g, og in zip(grads[li], ograds[li]):
            g = g.cpu().numpy().astype(np.float64).ravel()
            og = og.ravel()
            assert np.linalg.norm(g - og) <= 5e-2 * np.linalg.norm(og), li
            assert g @ og / (np.linalg.norm(g) * np.linalg.norm(og)) > 0.998, li


def test_adam_step(ws):
    import paper_2110_09667_gb300 as aa  # noqa: F401
    n = 1000
    w = aa_synth.normal(11, n).astype(np.float32)
    g = aa_synth.normal(12, n).astype(np.float32)
    W = torch.from_numpy(w.copy()).cuda()
    G = torch.from_numpy(g).cuda()
    m = torch.zeros(n, device="cuda")
    v = torch.zeros(n, device="cuda")
    Wb = torch.empty(n, dtype=torch.bfloat16, device="cuda")
    L = ws._L()
    for step in (1, 2):
        assert L.aa_adam(n, ws._p(W), ws._p(Wb), ws._p(G), ws._p(m), ws._p(v), 1e-2, 0.9, 0.999,
                         1e-8, step, 0.0, ws._stream()) == 0
    # reference (float64) for two steps with the same gradient
    mm = np.zeros(n)
    vv = np.zeros(n)
    ww = w.astype(np.float64)
    for step in (1, 2):
        mm = 0.9 * mm + 0.1 * g
        vv = 0.999 * vv + 0.001 * g.astype(np.float64) ** 2
        ww = ww - 1e-2 * (mm / (1 - 0.9 ** step)) / (np.sqrt(vv / (1 - 0.999 ** step)) + 1e-8)
    assert np.max(np.abs(W.cpu().numpy() - ww)) < 1e-5
    assert np.array_equal(Wb.float().cpu().numpy(), omlp.round_bf16(W.cpu().numpy()).astype(np.float32))


@pytest.mark.parametrize("impl", IMPLS)
def test_gemm_accumulate(ws, impl):
    """EPI_ACC: C += A B^T onto an FP32 C already in place (the output layer's
    second, low-order weight product)."""
    M, N, K = 50, 70, 48
    A = omlp.round_bf16(aa_synth.normal(21, M * K).reshape(M, K))
    B = omlp.round_bf16(aa_synth.normal(22, N * K).reshape(N, K))
    C0 = aa_synth.normal(23, M * N).reshape(M, N).astype(np.float32)
    C = torch.from_numpy(C0.copy()).cuda()
    ws.gemm_nt(bf16(A), bf16(B), C, epi=ws.EPI_ACC, impl=impl)
    _tc_ok(ws, impl)
    ref = C0.astype(np.float64) + A @ B.T
    bound = 2 * (K + 1) * 2.0 ** -24 * (np.abs(A) @ np.abs(B).T + np.abs(C0))
    assert np.all(np.abs(C.cpu().numpy() - ref) <= bound)


def test_sgd_step_and_split(ws):
    """Momentum SGD against float64 for two steps; the split copy satisfies
    hi = bf16(w), lo = bf16(w - hi), so |w - (hi + lo)| <= 2^-16 |w|."""
    n = 1000
    w = aa_synth.normal(31, n).astype(np.float32)
    g = aa_synth.normal(32, n).astype(np.float32)
    W = torch.from_numpy(w.copy()).cuda()
    G = torch.from_numpy(g).cuda()
    mom = torch.zeros(n, device="cuda")
    hi = torch.empty(n, dtype=torch.bfloat16, device="cuda")
    lo = torch.empty(n, dtype=torch.bfloat16, device="cuda")
    L = ws._L()
    for _ in range(2):
        assert L.aa_sgd(n, ws._p(W), ws._p(hi), ws._p(lo), ws._p(G), ws._p(mom), 0.05, 0.9, 0.0,
                        ws._stream()) == 0
    ww, mm = w.astype(np.float64), np.zeros(n)
    for _ in range(2):
        mm = 0.9 * mm + g
        ww = ww - 0.05 * mm
    wg = W.cpu().numpy()
    assert np.max(np.abs(wg - ww)) < 1e-5
    h = hi.float().cpu().numpy()
    lw = lo.float().cpu().numpy()
    assert np.array_equal(h, omlp.round_bf16(wg).astype(np.float32))
    assert np.array_equal(lw, omlp.round_bf16(wg.astype(np.float64) - h).astype(np.float32))
    assert np.all(np.abs(wg.astype(np.float64) - h - lw) <= 2.0 ** -16 * np.abs(wg))
    # the split conversion alone gives the same pair
    h2 = torch.empty_like(hi)
    l2 = torch.empty_like(lo)
    assert L.aa_f32_split_bf16(n, ws._p(W), ws._p(h2), ws._p(l2), ws._stream()) == 0
    assert torch.equal(h2, hi) and torch.equal(l2, lo)
