"""aa_mdot_noalloc, the allocation-free multi-dot, against aa_mdot.

Collected last on purpose (file name), so that a run stopping at its first
failure has run every other test already.  It must pass alone in a fresh
process (first call performs the per-device set-up) and after the others.
"""
import numpy as np
import pytest

import aa_synth

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu


def padded(rows, n, seed):
    ld = (n + 31) // 32 * 32  # 16-byte aligned columns
    t = torch.zeros(rows, ld, dtype=torch.float64, device="cuda")
    t[:, :n] = torch.from_numpy(aa_synth.uniform(seed, rows * n).reshape(rows, n)).cuda()
    return t[:, :n]


def test_noalloc_matches_mdot_two_calls():
    import paper_2110_09667_gb300 as aa
    n = (1 << 20) + 77  # several tiles and a ragged tail
    cases = [(padded(5, n, 1), padded(2, n, 2)), (padded(3, n, 3), padded(4, n, 4))]
    for A, V in cases:  # two calls in a row, different shapes and data
        k, nv = A.shape[0], V.shape[0]
        ref = aa.mdot(A, V)
        out = torch.full((k * nv,), float("nan"), dtype=torch.float64, device="cuda")
        aa.mdot_noalloc(A, V, out)
        torch.cuda.synchronize()
        got = out.cpu().numpy().reshape(k, nv)
        Ah, Vh = A.cpu().numpy(), V.cpu().numpy()
        scale = np.abs(Ah) @ np.abs(Vh).T
        assert np.all(np.abs(got - ref) <= 1e-14 * scale * np.log2(n))
        assert np.all(np.abs(got - Ah @ Vh.T) <= 1e-14 * scale * np.log2(n))


def test_noalloc_rejects_oversize():
    import paper_2110_09667_gb300 as aa
    n = 64
    A = padded(20, n, 5)
    V = padded(20, n, 6)  # 400 products > 256
    out = torch.empty(400, dtype=torch.float64, device="cuda")
    with pytest.raises(aa.AAError):
        aa.mdot_noalloc(A, V, out)


def test_noalloc_leaves_free_memory_unchanged():
    """The property the entry point exists for: after a first call (which
    looks up the scratch array's address and loads the kernel), further
    calls change the device's free memory by nothing."""
    import paper_2110_09667_gb300 as aa
    n = (1 << 18) + 5
    A, V = padded(4, n, 7), padded(3, n, 8)
    out = torch.empty(12, dtype=torch.float64, device="cuda")
    aa.mdot_noalloc(A, V, out)
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(5):
        aa.mdot_noalloc(A, V, out)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0, (free0, free1)
    ref = aa.mdot(A, V)
    assert np.allclose(out.cpu().numpy().reshape(4, 3), ref, rtol=1e-13, atol=0)
