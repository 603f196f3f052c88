"""The hot path at the benchmark's full size and launch configuration: 3D
7-point weighted Jacobi on 406^3 = 66,923,416 rows, AA(20), FP64 history,
every pass timed with CUDA events as the bench runs it.

The oracle cannot run 20 iterations at this size within a test, so the
checks are properties that hold at any size, against references that share
nothing with the kernels (cuSOLVER least squares and plain matrix products
through torch, FP64):
  - after the history is full (one recycle step with a QRDelete and a QRAdd),
    x_{i+1} = G(x_i) - dG gamma with gamma the least-squares solution of
    min ||f_i - F gamma|| (Algorithm 1, Algorithm 2), to the accuracy the
    conditioning of F allows;
  - the residual norm the step returns equals ||G(x_i) - x_i||.
"""
import numpy as np
import pytest

import aa_synth

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

NX = NY = NZ = 406
M = 20


@pytest.fixture(scope="module")
def aa():
    import paper_2110_09667_gb300 as aa
    aa.lib()
    return aa


def run(aa, orth, flags, extra_steps=2):
    n = NX * NY * NZ
    b = torch.from_numpy(aa_synth.jacobi3d_rhs(0, NX, NY, NZ)).cuda()
    P = aa.Jacobi3D(NX, NY, NZ, 0.1, 0.01, 0.8, b.data_ptr())
    gfn = aa.builtin_g("aa_g_jacobi3d")
    Pp = aa.C.cast(aa.C.pointer(P), aa.C.c_void_p)
    sp = torch.cuda.current_stream().cuda_stream
    A = aa.Anderson(n, M, orth, flags=aa.FLAG_TIMING | flags, max_iters=10**6)
    x = torch.zeros(n, dtype=torch.float64, device="cuda")
    xn = torch.empty_like(x)
    fs, gs = [], []
    for i in range(M + 1 + extra_steps):
        g = torch.empty_like(x)
        assert gfn(x.data_ptr(), g.data_ptr(), n, sp, Pp) == 0
        fn = A.step(x, g, xn)
        f = g - x
        assert abs(fn - float(torch.linalg.vector_norm(f))) <= 1e-12 * fn
        fs.append(f)
        gs.append(g)
        if len(fs) > M + 1:
            fs.pop(0)
            gs.pop(0)
        x, xn = xn, x
    # x is x_{i+1}; fs[-1], gs[-1] are f_i, G(x_i); the window holds M differences
    F = torch.stack([fs[j + 1] - fs[j] for j in range(M)], dim=1)
    dG = torch.stack([gs[j + 1] - gs[j] for j in range(M)], dim=1)
    del fs[:-1]
    gamma = torch.linalg.lstsq(F, fs[-1].unsqueeze(1)).solution.squeeze(1)
    Rr = torch.linalg.qr(F, mode="r").R
    sv = torch.linalg.svdvals(Rr)
    kappa = float(sv[0] / sv[-1])
    x_ref = gs[-1] - dG @ gamma
    err = float(torch.linalg.vector_norm(x - x_ref))
    scale = float(torch.linalg.vector_norm(dG) * torch.linalg.vector_norm(gamma))
    return err, scale, kappa, float(torch.linalg.vector_norm(x_ref)), A


@pytest.mark.parametrize("orth", ["mgs", "icwy", "cgs2", "dcgs2"])
def test_fullsize_recycle_step_fp64(aa, orth):
    flags = aa.FLAG_DCGS2_SCALED if orth == "dcgs2" else 0
    err, scale, kappa, xnorm, A = run(aa, orth, flags)
    # gamma errs by O(kappa eps) relative; the update adds O(eps) of ||x||
    tol = 64 * kappa * 2.0 ** -52 * scale + 1e-13 * xnorm
    assert err <= tol, (orth, err, tol, kappa)
    assert A.pass_times()  # the passes ran and were timed


def test_fullsize_recycle_step_df_arith(aa):
    """AA_FLAG_DF_ARITH at full size: (hi, lo) float arithmetic, 2^-48 per
    operation."""
    err, scale, kappa, xnorm, _ = run(aa, "icwy", aa.FLAG_DF_ARITH)
    tol = 64 * kappa * 2.0 ** -48 * scale + 1e-12 * xnorm
    assert err <= tol, (err, tol, kappa)
