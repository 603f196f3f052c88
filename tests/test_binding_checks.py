"""The Python binding checks every tensor before it passes a raw pointer to
the C ABI (which cannot see dtypes, strides or buffer sizes): wrong shapes,
strided views, short buffers, wrong dtypes and host tensors raise
ValueError before any device call.  Runs on the CPU: the checks come before
the library would touch the pointers."""
import pytest

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def aa():
    import paper_2110_09667_gb300 as aa
    aa.lib()
    return aa


def f64(*shape):
    return torch.zeros(*shape, dtype=torch.float64)


def test_mdot_shape_checks(aa):
    with pytest.raises(ValueError, match="2-D"):
        aa.mdot(f64(10), f64(2, 10))
    with pytest.raises(ValueError, match="entries per column"):
        aa.mdot(f64(3, 10), f64(2, 9))              # V shorter than A's columns
    with pytest.raises(ValueError, match="contiguous"):
        aa.mdot(f64(10, 3).t(), f64(2, 10))         # strided columns
    with pytest.raises(ValueError, match="empty"):
        aa.mdot(f64(0, 10), f64(2, 10))


def test_mdot_dtype_and_device_checks(aa):
    with pytest.raises(ValueError, match="float64"):
        aa.mdot(torch.zeros(3, 10, dtype=torch.float32), f64(2, 10))
    with pytest.raises(ValueError, match="CUDA"):
        aa.mdot(f64(3, 10), f64(2, 10))             # host tensors


def test_mdot_noalloc_output_checks(aa):
    A, V = f64(3, 10), f64(2, 10)
    with pytest.raises(ValueError, match="at least 6"):
        aa.mdot_noalloc(A, V, f64(5))               # out shorter than k * nv
    with pytest.raises(ValueError, match="unit stride"):
        aa.mdot_noalloc(A, V, f64(12)[::2])
    with pytest.raises(ValueError, match="float64"):
        aa.mdot_noalloc(A, V, torch.zeros(6, dtype=torch.float32))
    with pytest.raises(ValueError, match="CUDA"):
        aa.mdot_noalloc(A, V, f64(6))


def test_vector_checks(aa):
    with pytest.raises(ValueError, match="at least 8"):
        aa._vec(f64(7), 8, "x")
    with pytest.raises(ValueError, match="1-D"):
        aa._vec(f64(2, 4), 8, "x")
    with pytest.raises(ValueError, match="float64"):
        aa._vec(torch.zeros(8, dtype=torch.float32), 8, "x")
    with pytest.raises(ValueError, match="CUDA"):
        aa._vec(f64(8), 8, "x")


def test_gemm_checks(aa):
    from paper_2110_09667_gb300 import warmstart as ws
    bf = torch.bfloat16
    A, B = torch.zeros(4, 16, dtype=bf), torch.zeros(6, 16, dtype=bf)
    C = torch.zeros(4, 6)
    with pytest.raises(ValueError, match="columns"):
        ws.gemm_nt(A, torch.zeros(6, 8, dtype=bf), C)          # K mismatch
    with pytest.raises(ValueError, match="contiguous rows"):
        ws.gemm_nt(torch.zeros(16, 4, dtype=bf).t(), B, C)     # strided rows
    with pytest.raises(ValueError, match=r"\[4, 6\]"):
        ws.gemm_nt(A, B, torch.zeros(4, 5))                     # C too small
    with pytest.raises(ValueError, match="bias"):
        ws.gemm_nt(A, B, C, bias=torch.zeros(5), epi=ws.EPI_BIAS)
    with pytest.raises(ValueError, match="bfloat16"):
        ws.gemm_nt(A.float(), B, C)
    with pytest.raises(ValueError, match="C: expected torch.bfloat16"):
        ws.gemm_nt(A, B, C, epi=ws.EPI_BF16)                    # BF16 store into an FP32 C
    with pytest.raises(ValueError, match="CUDA"):
        ws.gemm_nt(A, B, C, impl="tc")                          # host tensors


def test_copy_checks(aa):
    a = torch.zeros(10, dtype=torch.float64)
    with pytest.raises(ValueError, match="sizes differ"):
        aa.copy(a, torch.zeros(9, dtype=torch.float64))
    with pytest.raises(ValueError, match="dtypes differ"):
        aa.copy(a, torch.zeros(10, dtype=torch.float32))
    with pytest.raises(ValueError, match="contiguous"):
        aa.copy(torch.zeros(20, dtype=torch.float64)[::2], a)
    with pytest.raises(ValueError, match="page-locked"):
        aa.copy(a, torch.zeros(10, dtype=torch.float64))        # pageable host tensors
