"""The hot path at the benchmark's full size and launch configuration: 3D
7-point weighted Jacobi on 406^3 = 66,923,416 rows, AA(20), FP64 history,
every pass timed with CUDA events as the bench runs it.

The oracle cannot run 20 iterations at this size within a test, so the
checks are properties that hold at any size, against references that share
nothing with the kernels (FP64 matrix products, Cholesky factors and
triangular solves through torch; CholeskyQR2 for the least-squares
reference):
  - after the history is full (one recycle step with a QRDelete and a QRAdd),
    x_{i+1} = G(x_i) - dG gamma with gamma the least-squares solution of
    min ||f_i - F gamma|| (Algorithm 1, Algorithm 2), to the accuracy the
    conditioning of F allows;
  - the residual norm the step returns equals ||G(x_i) - x_i||.
"""
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


def lstsq_cholqr2(Fr, f):
    """min ||f - F gamma|| for F with the columns given as the rows of Fr, by
    CholeskyQR2 (two Cholesky-QR passes; Yamamoto et al. 2015): accurate to
    O(kappa eps) while kappa^2 eps < 1.  FP64 matrix products (cuBLAS) and
    triangular solves only.  Returns gamma and the triangular factor R."""
    G1 = Fr @ Fr.T
    R1 = torch.linalg.cholesky(G1).T
    Q1 = torch.linalg.solve_triangular(R1.T, Fr, upper=False)
    R2 = torch.linalg.cholesky(Q1 @ Q1.T).T
    Q = torch.linalg.solve_triangular(R2.T, Q1, upper=False)
    del Q1
    R = R2 @ R1
    rhs = (Q @ f).unsqueeze(1)
    gamma = torch.linalg.solve_triangular(R, rhs, upper=True).squeeze(1)
    return gamma, R


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
    g = torch.empty_like(x)
    # the last M differences, one per row (ring), oldest at row `col` at the end
    Fr = torch.empty(M, n, dtype=torch.float64, device="cuda")
    Gr = torch.empty(M, n, dtype=torch.float64, device="cuda")
    f_prev = g_prev = None
    col = 0
    try:
        for i in range(M + 1 + extra_steps):
            assert gfn(x.data_ptr(), g.data_ptr(), n, sp, Pp) == 0
            fn = A.step(x, g, xn)
            f = g - x
            assert abs(fn - float(torch.linalg.vector_norm(f))) <= 1e-12 * fn
            if f_prev is not None:
                Fr[col] = f - f_prev
                Gr[col] = g - g_prev
                col = (col + 1) % M
            f_prev, g_prev = f, g.clone()
            x, xn = xn, x
        order = [(col + j) % M for j in range(M)]
        Fr, Gr = Fr[order], Gr[order]
        # x is x_{i+1}; f_prev, g_prev are f_i and G(x_i)
        gamma, R = lstsq_cholqr2(Fr, f_prev)
        sv = torch.linalg.svdvals(R)
        kappa = float(sv[0] / sv[-1])
        x_ref = g_prev - Gr.T @ gamma
        err = float(torch.linalg.vector_norm(x - x_ref))
        scale = float(torch.linalg.vector_norm(Gr) * torch.linalg.vector_norm(gamma))
        timed = bool(A.pass_times())
        return err, scale, kappa, float(torch.linalg.vector_norm(x_ref)), timed
    finally:
        del Fr, Gr, x, xn, g, f_prev, g_prev, A
        torch.cuda.empty_cache()


@pytest.mark.parametrize("orth", ["mgs", "icwy", "cgs2", "dcgs2"])
def test_fullsize_recycle_step_fp64(aa, orth):
    flags = aa.FLAG_DCGS2_SCALED if orth == "dcgs2" else 0
    err, scale, kappa, xnorm, timed = run(aa, orth, flags)
    # gamma errs by O(kappa eps) relative; the update adds O(eps) of ||x||
    tol = 64 * kappa * 2.0 ** -52 * scale + 1e-13 * xnorm
    assert err <= tol, (orth, err, tol, kappa)
    assert timed  # the passes ran and were timed


def test_fullsize_recycle_step_df_arith(aa):
    """AA_FLAG_DF_ARITH at full size: (hi, lo) float arithmetic, 2^-48 per
    operation."""
    err, scale, kappa, xnorm, _ = run(aa, "icwy", aa.FLAG_DF_ARITH)
    tol = 64 * kappa * 2.0 ** -48 * scale + 1e-12 * xnorm
    assert err <= tol, (err, tol, kappa)


@pytest.mark.parametrize("orth", ["icwy", "cgs2"])
def test_fullsize_recycle_step_fp32_dots(aa, orth):
    """AA_FLAG_FP32_DOTS at full size: FP32-pipe dot products in the first
    pass (and the CGS-2 middle pass), about 2^-46 of sum |a_i b_i| each."""
    err, scale, kappa, xnorm, _ = run(aa, orth, aa.FLAG_FP32_DOTS)
    tol = 64 * kappa * 2.0 ** -46 * scale + 1e-12 * xnorm
    assert err <= tol, (orth, err, tol, kappa)
