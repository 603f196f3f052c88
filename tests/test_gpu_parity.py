"""GPU parity: libaa's sm_103a path against the FP64 CPU oracle.

Every call goes through the C ABI (the ctypes binding only marshals
pointers).  Inputs are seeded (aa_synth); expected values come from the
oracle only.  Tolerances: FP64 iterates to relative 1e-10 over the first
20 iterations, iteration counts to +-1, QR factors to 1e-12 on
well-conditioned histories (the reduction order differs from the oracle's
sequential sums, nothing else).
"""
import numpy as np
import pytest

import aa_synth

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

VARIANTS = ["mgs", "icwy", "cgs2", "dcgs2"]


@pytest.fixture(scope="module")
def aa():
    import paper_2110_09667_gb300 as aa
    aa.lib()
    return aa


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()


# ----------------------------------------------------------------- mdot

@pytest.mark.parametrize("n", [1, 7, 33, 4097, 1 << 20])
def test_mdot_matches_dot(aa, n):
    k, nv = 5, 2
    A = aa_synth.uniform(1, k * n).reshape(k, n)
    V = aa_synth.uniform(2, nv * n).reshape(nv, n)
    ld = (n + 31) // 32 * 32  # columns must start 16-byte aligned
    Ad = torch.zeros(k, ld, dtype=torch.float64, device="cuda")
    Vd = torch.zeros(nv, ld, dtype=torch.float64, device="cuda")
    Ad[:, :n] = dev(A)
    Vd[:, :n] = dev(V)
    got = aa.mdot(Ad[:, :n], Vd[:, :n])
    ref = A @ V.T
    scale = np.abs(A) @ np.abs(V).T
    assert np.all(np.abs(got - ref) <= 1e-14 * scale * max(1.0, np.log2(n)))
    # deterministic two-stage reduction: bit-identical on repeat
    got2 = aa.mdot(Ad[:, :n], Vd[:, :n])
    assert np.array_equal(got, got2)


# ----------------------------------------------------------- QR updates

@pytest.mark.parametrize("orth", VARIANTS)
@pytest.mark.parametrize("m", [1, 3, 5])
@pytest.mark.parametrize("n", [1, 7, 33, 4097])
def test_qradd_matches_oracle(aa, ora, orth, m, n):
    if n < m + 3:  # need full-rank histories
        pytest.skip("history longer than n")
    adds = m + 4  # several deletes
    V = aa_synth.uniform(10 + m, adds * n).reshape(adds, n)
    O = ora.Oracle(n, m, orth)
    G = aa.Anderson(n, m, orth)
    for j in range(adds):
        assert O.qradd(V[j]) == ora.OK
        assert G.qradd(dev(V[j])) == 0
        Qo, Ro, To = O.get_qr()
        Qg, Rg, Tg = G.get_qr()
        assert Qg.shape == Qo.shape
        tol = 1e-11 if orth != "dcgs2" else 1e-9
        assert np.max(np.abs(Rg - Ro)) <= tol * np.abs(Ro).max(), (j, orth)
        assert np.max(np.abs(Qg - Qo)) <= tol, (j, orth)
        if orth == "icwy" and Qo.shape[1] >= 2:
            assert np.max(np.abs(Tg[:-1] - To[:-1])) <= 1e-11


@pytest.mark.parametrize("orth", VARIANTS)
def test_lsq_matches_oracle(aa, ora, orth):
    n, m = 4097, 5
    V = aa_synth.uniform(20, 8 * n).reshape(8, n)
    f = aa_synth.uniform(21, n)
    O = ora.Oracle(n, m, orth)
    G = aa.Anderson(n, m, orth)
    for j in range(8):
        O.qradd(V[j])
        G.qradd(dev(V[j]))
    go = O.lsq(f)
    gg = G.lsq(dev(f))
    assert np.max(np.abs(gg - go)) <= 1e-11 * np.abs(go).max()


@pytest.mark.parametrize("orth", VARIANTS)
def test_breakdown_clears(aa, orth):
    n, m = 300, 4
    V = aa_synth.uniform(30, 3 * n).reshape(3, n)
    G = aa.Anderson(n, m, orth)
    for j in range(3):
        G.qradd(dev(V[j]))
    rc = G.qradd(dev(V.T @ np.array([1.0, -2.0, 0.5])))
    assert rc == aa.AA_EBREAKDOWN
    _, R, _ = G.get_qr()
    assert R.shape == (0, 0)
    assert G.qradd(dev(V[0])) == 0


# -------------------------------------------------------------- AA steps

def run_steps(aa, ora, Gmap, n, m, orth, iters, storage="fp64", **kw):
    O = ora.Oracle(n, m, orth, store_round={"fp64": 0, "fp32": 1, "bf16": 2}[storage])
    A = aa.Anderson(n, m, orth, storage, **kw)
    x_o = np.zeros(n)
    x_g = torch.zeros(n, dtype=torch.float64, device="cuda")
    xn_g = torch.empty_like(x_g)
    out = []
    for i in range(iters):
        g_o = Gmap(x_o)
        xn_o, fo, st = O.step(x_o, g_o)
        g_g = dev(Gmap(x_g.cpu().numpy()))
        fg = A.step(x_g, g_g, xn_g)
        out.append((xn_o.copy(), xn_g.cpu().numpy(), fo, fg))
        x_o = xn_o
        x_g, xn_g = xn_g, x_g
    return out, A


@pytest.mark.parametrize("orth", VARIANTS)
@pytest.mark.parametrize("m", [1, 5, 10])
def test_step_parity_jacobi2d(aa, ora, orth, m):
    """First 20 iterates of the 64 x 64 anisotropic Jacobi problem."""
    nx = ny = 64
    b = aa_synth.jacobi2d_rhs(0, nx, ny)
    Gmap = lambda x: ora.g_jacobi2d(nx, ny, 0.01, b, x)
    out, A = run_steps(aa, ora, Gmap, nx * ny, m, orth, 21)
    for i, (xo, xg, fo, fg) in enumerate(out):
        assert abs(fg - fo) <= 1e-10 * abs(fo), (i, fo, fg)
        assert np.linalg.norm(xg - xo) <= 1e-10 * np.linalg.norm(xo), (i, orth, m)


@pytest.mark.parametrize("orth", VARIANTS)
def test_step_parity_bratu_ragged(aa, ora, orth):
    """Nonlinear map on a ragged size (n = 45^2 = 2025, not a tile multiple)."""
    s, lam = 45, 5.0
    Gmap = lambda u: ora.g_bratu2d(s, lam, None, u)
    out, _ = run_steps(aa, ora, Gmap, s * s, 4, orth, 20)
    for i, (xo, xg, fo, fg) in enumerate(out):
        assert np.linalg.norm(xg - xo) <= 1e-10 * np.linalg.norm(xo), (i, orth)


@pytest.mark.parametrize("orth", VARIANTS)
def test_solve_jacobi2d_64_to_tol(aa, ora, orth):
    """The 64 x 64 workload to ||f||/||b|| < 1e-8: same iteration count (+-1)
    and the same solution."""
    nx = ny = 64
    n = nx * ny
    b = aa_synth.jacobi2d_rhs(0, nx, ny)
    scale = float(np.linalg.norm(b))
    O = ora.Oracle(n, 5, orth)
    ro = O.solve({"kind": "jacobi2d", "nx": nx, "ny": ny, "eps": 0.01, "b": b}, np.zeros(n),
                 max_iters=500, tol=1e-8, scale=scale)
    A = aa.Anderson(n, 5, orth, tol=1e-8, scale=scale, max_iters=500)
    bd = dev(b)
    P = aa.Jacobi2D(nx, ny, 0.01, bd.data_ptr())
    x = torch.zeros(n, dtype=torch.float64, device="cuda")
    rc, st = A.solve(aa.builtin_g("aa_g_jacobi2d"), P, x)
    assert (rc == 0) == (ro["status"] == 0)
    assert abs(st["iters"] - ro["iters"]) <= 1, (st["iters"], ro["iters"])
    xg = x.cpu().numpy()
    res = np.linalg.norm(ora.g_jacobi2d(nx, ny, 0.01, b, xg) - xg) / scale
    if ro["status"] == 0:
        assert res < 1.01e-8
        assert np.linalg.norm(xg - ro["x"]) <= 1e-6 * np.linalg.norm(ro["x"])


@pytest.mark.parametrize("orth,startup,recycle", [
    ("mgs", lambda mi: mi, lambda m: m),
    ("icwy", lambda mi: 2 if mi > 1 else 1, lambda m: 2),
    ("cgs2", lambda mi: 3 if mi > 1 else 1, lambda m: 3),
    ("dcgs2", lambda mi: 2 if mi > 1 else 1, lambda m: 2),
])
def test_gpu_reduction_counts(aa, orth, startup, recycle):
    """Grid-wide reduction passes per QRAdd.  Start-up matches the paper's
    tallies (Sec. 4.1); at recycle ICWY needs 2 here because the correction
    matrix is rotated at the m x m level instead of re-reduced."""
    n, m = 1000, 6
    V = aa_synth.uniform(40, (m + 3) * n).reshape(m + 3, n)
    A = aa.Anderson(n, m, orth)
    for j in range(m + 3):
        before = A.stats()["reductions"]
        A.qradd(dev(V[j]))
        d = A.stats()["reductions"] - before
        if j < m:
            assert d == startup(j + 1), (j, d)
        else:
            assert d == recycle(m), (j, d)


def test_nonfinite_reported(aa):
    n = 100
    A = aa.Anderson(n, 3, "mgs")
    x = torch.zeros(n, dtype=torch.float64, device="cuda")
    g = torch.ones(n, dtype=torch.float64, device="cuda")
    xn = torch.empty_like(x)
    A.step(x, g, xn)
    g2 = g.clone()
    g2[5] = float("nan")
    with pytest.raises(aa.AAError) as e:
        A.step(xn, g2, x)
    assert e.value.code == -5


def test_stagnation_breakdown_falls_back(aa, ora):
    """f_i == f_{i-1} makes Delta f = 0: the step restarts the history and
    returns x_{i+1} = G(x_i), as the oracle does."""
    n = 64
    O = ora.Oracle(n, 3, "icwy")
    A = aa.Anderson(n, 3, "icwy")
    x = aa_synth.uniform(50, n)
    g = x + 1.0
    xo1, _, _ = O.step(x, g)
    xo2, _, st = O.step(x + 0.0, g)
    assert st == ora.BREAKDOWN
    xg = torch.empty(n, dtype=torch.float64, device="cuda")
    A.step(dev(x), dev(g), xg)
    A.step(dev(x), dev(g), xg)
    assert A.stats()["breakdowns"] == 1
    assert np.array_equal(xg.cpu().numpy(), xo2)


# ------------------------------------- FP64 storage, FP32-pipe dot products

@pytest.mark.parametrize("orth", VARIANTS)
def test_step_parity_fp32_dots(aa, ora, orth):
    """AA_FLAG_FP32_DOTS keeps the FP64 parity contract: the dot products of
    passes with more than four of them are formed on the FP32 pipe from
    scaled (hi, lo) splits (exact head products, compensated float-pair
    sums over 64 rows per lane, error about 2^-46 of sum |a_i b_i|) and
    accumulated in FP64; squared norms stay FP64."""
    nx = ny = 64
    b = aa_synth.jacobi2d_rhs(0, nx, ny)
    Gmap = lambda x: ora.g_jacobi2d(nx, ny, 0.01, b, x)
    out, _ = run_steps(aa, ora, Gmap, nx * ny, 5, orth, 21, flags=aa.FLAG_FP32_DOTS)
    for i, (xo, xg, fo, fg) in enumerate(out):
        assert abs(fg - fo) <= 1e-10 * abs(fo), (i, fo, fg)
        assert np.linalg.norm(xg - xo) <= 1e-10 * np.linalg.norm(xo), (i, orth)


@pytest.mark.parametrize("orth", VARIANTS)
def test_qradd_fp32_dots(aa, ora, orth):
    n, m = 4097, 4
    V = aa_synth.uniform(60, (m + 4) * n).reshape(m + 4, n)
    O = ora.Oracle(n, m, orth)
    G = aa.Anderson(n, m, orth, flags=aa.FLAG_FP32_DOTS)
    for j in range(m + 4):
        O.qradd(V[j])
        G.qradd(dev(V[j]))
        Qo, Ro, _ = O.get_qr()
        Qg, Rg, _ = G.get_qr()
        tol = 1e-11 if orth != "dcgs2" else 1e-9
        assert np.max(np.abs(Rg - Ro)) <= tol * np.abs(Ro).max(), (j, orth)
        assert np.max(np.abs(Qg - Qo)) <= tol, (j, orth)


@pytest.mark.parametrize("orth", VARIANTS)
def test_step_parity_fp32_dots_m20(aa, ora, orth):
    """AA_FLAG_FP32_DOTS at the bench's history depth: 30 iterates, 10 of them
    with a delete, to the FP64 contract."""
    nx = ny = 64
    b = aa_synth.jacobi2d_rhs(0, nx, ny)
    Gmap = lambda x: ora.g_jacobi2d(nx, ny, 0.01, b, x)
    out, _ = run_steps(aa, ora, Gmap, nx * ny, 20, orth, 30, flags=aa.FLAG_FP32_DOTS)
    for i, (xo, xg, fo, fg) in enumerate(out):
        assert abs(fg - fo) <= 1e-10 * abs(fo), (i, fo, fg)
        assert np.linalg.norm(xg - xo) <= 1e-10 * np.linalg.norm(xo), (i, orth)


@pytest.mark.parametrize("orth", VARIANTS)
@pytest.mark.parametrize("m", [20, 50])
def test_qradd_fp32_dots_deep(aa, ora, orth, m):
    """QR factors with FP32-pipe dot products after m + 6 adds, ragged n:
    the exact form's tolerance, 1e-11 (DCGS-2 1e-9); measured at m = 20, 50,
    64: R to 2.3e-15 relative, Q to 1.3e-16."""
    n = 4097
    V = aa_synth.uniform(80 + m, (m + 6) * n).reshape(m + 6, n)
    O = ora.Oracle(n, m, orth)
    G = aa.Anderson(n, m, orth, flags=aa.FLAG_FP32_DOTS)
    for j in range(m + 6):
        O.qradd(V[j])
        G.qradd(dev(V[j]))
    Qo, Ro, _ = O.get_qr()
    Qg, Rg, _ = G.get_qr()
    tol = 1e-11 if orth != "dcgs2" else 1e-9
    assert np.max(np.abs(Rg - Ro)) <= tol * np.abs(Ro).max(), orth
    assert np.max(np.abs(Qg - Qo)) <= tol, orth


@pytest.mark.parametrize("orth", ["icwy", "cgs2"])
@pytest.mark.parametrize("scale", [1e-30, 1e30])
def test_qradd_fp32_dots_far_from_one(aa, ora, orth, scale):
    """Inputs far outside the float range's comfortable middle: the operands
    of the FP32-pipe products are scaled by powers of two (exact) chosen from
    the previous norms, so tiny and huge columns give the oracle's factors
    (R scales with the input, Q does not)."""
    n, m = 4097, 6
    V = scale * aa_synth.uniform(90, (m + 3) * n).reshape(m + 3, n)
    O = ora.Oracle(n, m, orth)
    G = aa.Anderson(n, m, orth, flags=aa.FLAG_FP32_DOTS)
    for j in range(m + 3):
        O.qradd(V[j])
        G.qradd(dev(V[j]))
        Qo, Ro, _ = O.get_qr()
        Qg, Rg, _ = G.get_qr()
        assert np.max(np.abs(Rg - Ro)) <= 1e-11 * np.abs(Ro).max(), (j, orth)
        assert np.max(np.abs(Qg - Qo)) <= 1e-11, (j, orth)


# ------------------------- FP64 storage, (hi, lo) float arithmetic (MODE 3)

@pytest.mark.parametrize("orth", VARIANTS)
@pytest.mark.parametrize("m", [5, 10])
def test_step_parity_df_arith(aa, ora, orth, m):
    """AA_FLAG_DF_ARITH keeps the FP64 parity contract (iterates to 1e-10 over
    20 iterations): every n-space operation errs by about 2^-48 relative
    instead of 2^-53."""
    nx = ny = 64
    b = aa_synth.jacobi2d_rhs(0, nx, ny)
    Gmap = lambda x: ora.g_jacobi2d(nx, ny, 0.01, b, x)
    out, _ = run_steps(aa, ora, Gmap, nx * ny, m, orth, 21, flags=aa.FLAG_DF_ARITH)
    for i, (xo, xg, fo, fg) in enumerate(out):
        assert abs(fg - fo) <= 1e-10 * abs(fo), (i, fo, fg)
        assert np.linalg.norm(xg - xo) <= 1e-10 * np.linalg.norm(xo), (i, orth, m)


@pytest.mark.parametrize("orth", VARIANTS)
def test_step_parity_df_arith_bratu_ragged(aa, ora, orth):
    s, lam = 45, 5.0
    Gmap = lambda u: ora.g_bratu2d(s, lam, None, u)
    out, _ = run_steps(aa, ora, Gmap, s * s, 4, orth, 20, flags=aa.FLAG_DF_ARITH)
    for i, (xo, xg, fo, fg) in enumerate(out):
        assert np.linalg.norm(xg - xo) <= 1e-10 * np.linalg.norm(xo), (i, orth)


@pytest.mark.parametrize("orth", VARIANTS)
@pytest.mark.parametrize("n", [7, 4097])
def test_qradd_df_arith(aa, ora, orth, n):
    m = 4
    V = aa_synth.uniform(61, (m + 4) * n).reshape(m + 4, n)
    O = ora.Oracle(n, m, orth)
    G = aa.Anderson(n, m, orth, flags=aa.FLAG_DF_ARITH)
    for j in range(m + 4):
        O.qradd(V[j])
        G.qradd(dev(V[j]))
        Qo, Ro, _ = O.get_qr()
        Qg, Rg, _ = G.get_qr()
        tol = 1e-11 if orth != "dcgs2" else 1e-9
        assert np.max(np.abs(Rg - Ro)) <= tol * np.abs(Ro).max(), (j, orth)
        assert np.max(np.abs(Qg - Qo)) <= tol, (j, orth)


def test_lsq_df_arith(aa, ora):
    n, m = 3001, 6
    V = aa_synth.uniform(62, (m + 1) * n).reshape(m + 1, n)
    O = ora.Oracle(n, m, "icwy")
    G = aa.Anderson(n, m, "icwy", flags=aa.FLAG_DF_ARITH)
    for j in range(m):
        O.qradd(V[j])
        G.qradd(dev(V[j]))
    go = O.lsq(V[m])
    gg = G.lsq(dev(V[m]))
    assert np.max(np.abs(gg - go)) <= 1e-11 * np.abs(go).max()


def test_df_arith_rejects_other_modes(aa):
    with pytest.raises(aa.AAError):
        aa.Anderson(100, 3, "icwy", "fp32", flags=aa.FLAG_DF_ARITH)
    with pytest.raises(aa.AAError):
        aa.Anderson(100, 3, "icwy", flags=aa.FLAG_DF_ARITH | aa.FLAG_FP32_DOTS)


# ------------------------------------------- deep histories (the bench's m)

@pytest.mark.parametrize("orth", VARIANTS)
@pytest.mark.parametrize("m", [20, 50, 64])
def test_qradd_deep_history(aa, ora, orth, m):
    """QR factors after m + 6 adds (6 deletes) for the bench's history depths
    and the largest one the library takes (64), on a ragged n.  The inputs
    are well conditioned (independent uniform vectors), so the factors agree
    to the same tolerance as at small m: 1e-11 (DCGS-2 1e-9), the bound that
    holds at every m here (measured at m = 20, 50, 64: R to 3e-15 relative,
    Q to 1.3e-16)."""
    n = 4097
    V = aa_synth.uniform(70 + m, (m + 6) * n).reshape(m + 6, n)
    O = ora.Oracle(n, m, orth)
    G = aa.Anderson(n, m, orth)
    for j in range(m + 6):
        O.qradd(V[j])
        G.qradd(dev(V[j]))
    Qo, Ro, _ = O.get_qr()
    Qg, Rg, _ = G.get_qr()
    tol = 1e-11 if orth != "dcgs2" else 1e-9
    assert np.max(np.abs(Rg - Ro)) <= tol * np.abs(Ro).max(), orth
    assert np.max(np.abs(Qg - Qo)) <= tol, orth
    if orth != "dcgs2":  # the literal DCGS-2 update is checked against the oracle only
        assert np.max(np.abs(Qg.T @ Qg - np.eye(m))) <= 1e-12


@pytest.mark.parametrize("orth", VARIANTS)
def test_step_parity_jacobi2d_m20(aa, ora, orth):
    """The bench's history depth on the 64 x 64 problem: 30 iterates
    (10 with a delete)."""
    nx = ny = 64
    b = aa_synth.jacobi2d_rhs(0, nx, ny)
    Gmap = lambda x: ora.g_jacobi2d(nx, ny, 0.01, b, x)
    out, _ = run_steps(aa, ora, Gmap, nx * ny, 20, orth, 30)
    for i, (xo, xg, fo, fg) in enumerate(out):
        assert abs(fg - fo) <= 1e-10 * abs(fo), (i, fo, fg)
        assert np.linalg.norm(xg - xo) <= 1e-10 * np.linalg.norm(xo), (i, orth)


def test_create_rejects_bad_sizes(aa):
    """Empty and oversized inputs are refused before any device work."""
    with pytest.raises(aa.AAError):
        aa.Anderson(0, 5, "icwy")
    with pytest.raises(aa.AAError):
        aa.Anderson(100, 65, "icwy")
    with pytest.raises(aa.AAError):
        aa.Anderson(100, 0, "icwy")


def test_solve_python_callback_and_callback_error(aa, ora):
    """aa_solve over a G written in Python (it forwards to the built-in 2D map
    and counts its calls): the iterates equal those of the built-in callback;
    a callback that returns non-zero stops the solve with AA_ECALLBACK after
    exactly that call."""
    nx = ny = 32
    n = nx * ny
    b = aa_synth.jacobi2d_rhs(0, nx, ny)
    bd = dev(b)
    P = aa.Jacobi2D(nx, ny, 0.01, bd.data_ptr())
    inner = aa.builtin_g("aa_g_jacobi2d")
    calls = []

    def make(fail_at):
        @aa.GFN
        def g(x, gx, nn, stream, user):
            calls.append(1)
            if len(calls) == fail_at:
                return 3
            return inner(x, gx, nn, stream, user)
        return g

    A1 = aa.Anderson(n, 5, "icwy", max_iters=30, tol=1e-30)
    x1 = torch.zeros(n, dtype=torch.float64, device="cuda")
    rc1, st1 = A1.solve(inner, P, x1)
    calls.clear()
    g_ok = make(-1)
    A2 = aa.Anderson(n, 5, "icwy", max_iters=30, tol=1e-30)
    x2 = torch.zeros(n, dtype=torch.float64, device="cuda")
    rc2, st2 = A2.solve(g_ok, P, x2)
    assert rc1 == rc2 and st1["iters"] == st2["iters"]
    assert torch.equal(x1, x2)
    calls.clear()
    g_bad = make(4)
    A3 = aa.Anderson(n, 5, "icwy", max_iters=30, tol=1e-30)
    x3 = torch.zeros(n, dtype=torch.float64, device="cuda")
    with pytest.raises(aa.AAError) as e:
        A3.solve(g_bad, P, x3)
    assert e.value.code == -7
    assert len(calls) == 4


# ------------------------------------------------------- built-in maps G

@pytest.mark.parametrize("shape", [(1, 1), (37, 23), (64, 64), (130, 5)])
def test_builtin_jacobi2d_matches_oracle(aa, ora, shape):
    """The device map evaluates G = x + D^{-1}(b - A x) with the diagonal
    term cancelled; it equals the oracle's literal form to a few roundings."""
    nx, ny = shape
    n = nx * ny
    b = aa_synth.jacobi2d_rhs(3, nx, ny)
    x = aa_synth.uniform(4, n)
    bd, xd = dev(b), dev(x)
    gd = torch.empty_like(xd)
    P = aa.Jacobi2D(nx, ny, 0.01, bd.data_ptr())
    rc = aa.builtin_g("aa_g_jacobi2d")(xd.data_ptr(), gd.data_ptr(), n,
                                         torch.cuda.current_stream().cuda_stream,
                                         aa.C.cast(aa.C.pointer(P), aa.C.c_void_p))
    assert rc == 0
    ref = ora.g_jacobi2d(nx, ny, 0.01, b, x)
    scale = np.abs(x).max() + np.abs(b).max()
    assert np.max(np.abs(gd.cpu().numpy() - ref)) <= 1e-14 * scale


@pytest.mark.parametrize("shape", [(1, 1, 1), (19, 13, 7), (33, 2, 40), (406, 406, 3)])
def test_builtin_jacobi3d_matches_oracle(aa, ora, shape):
    """The bench's map, (1 - omega) x + (omega/d)(b + neighbour sums), against
    the oracle's x + omega D^{-1}(b - A x), ragged sizes and the bench's plane."""
    nx, ny, nz = shape
    n = nx * ny * nz
    b = aa_synth.jacobi3d_rhs(5, nx, ny, nz)
    x = aa_synth.uniform(6, n)
    bd, xd = dev(b), dev(x)
    gd = torch.empty_like(xd)
    P = aa.Jacobi3D(nx, ny, nz, 0.1, 0.01, 0.8, bd.data_ptr())
    rc = aa.builtin_g("aa_g_jacobi3d")(xd.data_ptr(), gd.data_ptr(), n,
                                         torch.cuda.current_stream().cuda_stream,
                                         aa.C.cast(aa.C.pointer(P), aa.C.c_void_p))
    assert rc == 0
    ref = ora.g_jacobi3d(nx, ny, nz, 0.1, 0.01, 0.8, b, x)
    scale = np.abs(x).max() + np.abs(b).max()
    assert np.max(np.abs(gd.cpu().numpy() - ref)) <= 1e-14 * scale


@pytest.mark.parametrize("s,with_src", [(1, False), (45, False), (45, True), (130, True)])
def test_builtin_bratu2d_matches_oracle(aa, ora, s, with_src):
    n = s * s
    u = 0.5 * aa_synth.uniform(7, n)
    src = aa_synth.uniform(8, n) if with_src else None
    ud = dev(u)
    sd = dev(src) if with_src else None
    gd = torch.empty_like(ud)
    P = aa.Bratu2D(s, 5.0, sd.data_ptr() if with_src else None)
    rc = aa.builtin_g("aa_g_bratu2d")(ud.data_ptr(), gd.data_ptr(), n,
                                        torch.cuda.current_stream().cuda_stream,
                                        aa.C.cast(aa.C.pointer(P), aa.C.c_void_p))
    assert rc == 0
    ref = ora.g_bratu2d(s, 5.0, src, u)
    assert np.max(np.abs(gd.cpu().numpy() - ref)) <= 1e-14 * (np.abs(ref).max() + 1.0)


def test_builtin_map_rejects_wrong_size(aa):
    b = torch.zeros(12, dtype=torch.float64, device="cuda")
    P = aa.Jacobi3D(2, 2, 3, 0.1, 0.01, 0.8, b.data_ptr())
    rc = aa.builtin_g("aa_g_jacobi3d")(b.data_ptr(), b.data_ptr(), 13,
                                         torch.cuda.current_stream().cuda_stream,
                                         aa.C.cast(aa.C.pointer(P), aa.C.c_void_p))
    assert rc == -1  # AA_EINVAL
