"""Precision form: Q and dG stored in FP32 (or BF16), everything else FP64.

Parity is against the oracle with the same storage rounding (store_round),
so both sides round the same quantities to the storage type; they round at
slightly different points (the GPU stores v / ||Delta f|| with a column
scale, the oracle stores v / rho), so stored entries may differ by one unit
in the last place of the storage type.  Tolerances follow from that:
FP32 -- 2^-24 per stored entry times the conditioning of the small
least-squares problem over 20 iterations (< 1e3) gives 1e-4 relative on the
iterates; BF16 -- 2^-8 per entry, checked only for convergence behaviour.
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


def steps(aa, ora, Gmap, n, m, orth, iters, storage):
    O = ora.Oracle(n, m, orth, store_round={"fp64": 0, "fp32": 1, "bf16": 2}[storage])
    A = aa.Anderson(n, m, orth, storage)
    x_o = np.zeros(n)
    x_g = torch.zeros(n, dtype=torch.float64, device="cuda")
    xn_g = torch.empty_like(x_g)
    out = []
    for _ in range(iters):
        xn_o, fo, _ = O.step(x_o, Gmap(x_o))
        fg = A.step(x_g, dev(Gmap(x_g.cpu().numpy())), xn_g)
        out.append((xn_o.copy(), xn_g.cpu().numpy(), fo, fg))
        x_o = xn_o
        x_g, xn_g = xn_g, x_g
    return out, A


@pytest.mark.parametrize("orth", VARIANTS)
def test_fp32_storage_parity(aa, ora, orth):
    nx = ny = 64
    b = aa_synth.jacobi2d_rhs(0, nx, ny)
    Gmap = lambda x: ora.g_jacobi2d(nx, ny, 0.01, b, x)
    out, A = steps(aa, ora, Gmap, nx * ny, 5, orth, 21, "fp32")
    for i, (xo, xg, fo, fg) in enumerate(out):
        assert np.linalg.norm(xg - xo) <= 1e-4 * np.linalg.norm(xo), (i, orth)
    Q, R, _ = A.get_qr()
    loss = np.linalg.norm(np.eye(Q.shape[1]) - Q.T @ Q)
    # stored in FP32: orthogonality at the FP32 level, not worse
    assert loss < 1e-5, loss


def converge(aa, n, m, orth, storage, gname, P, scale, max_iters):
    A = aa.Anderson(n, m, orth, storage, tol=1e-8, scale=scale, max_iters=max_iters)
    x = torch.zeros(n, dtype=torch.float64, device="cuda")
    rc, st = A.solve(aa.builtin_g(gname), P, x)
    return rc, st, x.cpu().numpy()


@pytest.mark.parametrize("orth", ["icwy", "cgs2"])
def test_fp32_storage_reaches_1e8(aa, ora, orth):
    """3D weighted Jacobi 32^3, AA(20): the FP32-history form reaches
    ||f||/||b|| < 1e-8 like the FP64 form, to the same solution."""
    nx = ny = nz = 32
    n = nx * ny * nz
    b = aa_synth.jacobi3d_rhs(0, nx, ny, nz)
    scale = float(np.linalg.norm(b))
    bd = dev(b)
    P = aa.Jacobi3D(nx, ny, nz, 0.1, 0.01, 0.8, bd.data_ptr())
    rc64, st64, x64 = converge(aa, n, 20, orth, "fp64", "aa_g_jacobi3d", P, scale, 2000)
    rc32, st32, x32 = converge(aa, n, 20, orth, "fp32", "aa_g_jacobi3d", P, scale, 2000)
    assert rc64 == 0 and rc32 == 0
    res = np.linalg.norm(ora.g_jacobi3d(nx, ny, nz, 0.1, 0.01, 0.8, b, x32) - x32) / scale
    assert res < 1.01e-8
    assert np.linalg.norm(x32 - x64) <= 1e-6 * np.linalg.norm(x64)
    assert st32["iters"] <= 1.5 * st64["iters"] + 10


def test_bf16_storage_probe(aa, ora):
    """BF16 history storage (probe): the iteration still converges on the
    small 3D problem; no parity claim beyond that."""
    nx = ny = nz = 16
    n = nx * ny * nz
    b = aa_synth.jacobi3d_rhs(0, nx, ny, nz)
    scale = float(np.linalg.norm(b))
    bd = dev(b)
    P = aa.Jacobi3D(nx, ny, nz, 0.1, 0.01, 0.8, bd.data_ptr())
    rc, st, x = converge(aa, n, 10, "cgs2", "bf16", "aa_g_jacobi3d", P, scale, 5000)
    res = np.linalg.norm(ora.g_jacobi3d(nx, ny, nz, 0.1, 0.01, 0.8, b, x) - x) / scale
    assert rc == 0 and res < 1.01e-8


@pytest.mark.parametrize("m", [5, 10, 20])
@pytest.mark.parametrize("orth", VARIANTS)
def test_fp32_storage_qradd_multitile(aa, ora, orth, m):
    """QRAdd alone (the first pass in its unit-vector form, plus the
    projection) with FP32 history, at m = 5, 10 and 20 (both slot buckets of
    the column-family dot phase) on 300,001 rows (1,172 tiles: several per
    CTA, a ragged last tile): Q and R after m + 3 adds (three deletes) against
    the oracle with the same FP32 storage rounding.  Stored entries may differ
    by an FP32 unit where the two sides round at different points, and the
    device rotates in FP32 (float multipliers), so the bound is 1e-4 of the largest
    entry."""
    n = 300_001
    adds = m + 3
    V = aa_synth.uniform(70 + m, adds * n).reshape(adds, n)
    O = ora.Oracle(n, m, orth, store_round=1)
    G = aa.Anderson(n, m, orth, "fp32")
    for j in range(adds):
        assert O.qradd(V[j]) == ora.OK
        assert G.qradd(dev(V[j])) == 0
    Qo, Ro, _ = O.get_qr()
    Qg, Rg, _ = G.get_qr()
    assert Qg.shape == Qo.shape
    assert np.max(np.abs(Rg - Ro)) <= 1e-4 * np.abs(Ro).max(), orth
    assert np.max(np.abs(Qg - Qo)) <= 1e-4 * np.abs(Qo).max(), orth


@pytest.mark.parametrize("m", [3, 8])
@pytest.mark.parametrize("orth", ["icwy", "mgs"])
def test_fp32_storage_lsq(aa, ora, orth, m):
    """The least-squares solve R gamma = Q^T f alone (aa_lsq) with FP32
    history, after m + 2 adds on 70,001 rows: m = 3 takes its dot products
    as FP64 row sums (at most four of them), m = 8 through the dot phase.
    gamma against the oracle with the same FP32 storage rounding."""
    n = 70_001
    V = aa_synth.uniform(90 + m, (m + 2) * n).reshape(m + 2, n)
    f = aa_synth.uniform(91 + m, n)
    O = ora.Oracle(n, m, orth, store_round=1)
    G = aa.Anderson(n, m, orth, "fp32")
    for j in range(m + 2):
        assert O.qradd(V[j]) == ora.OK
        assert G.qradd(dev(V[j])) == 0
    go = O.lsq(f)
    gg = G.lsq(dev(f))
    assert np.max(np.abs(gg - go)) <= 1e-4 * np.abs(go).max(), (orth, m)
