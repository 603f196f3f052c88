"""aa_copy: the copy kernel between page-locked host memory and the device
(and device to device), bit-exact, with sizes that leave a tail of fewer than
16 bytes; pageable host memory goes through the cudaMemcpyAsync path."""
import ctypes as C

import numpy as np
import pytest

import aa_synth

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def aa():
    import paper_2110_09667_gb300 as aa
    aa.lib()
    return aa


@pytest.mark.parametrize("n", [1, 3, 1000003, 8_000_017])
def test_copy_pinned_roundtrip(aa, n):
    h = torch.from_numpy(aa_synth.uniform(5, n)).pin_memory()
    d = torch.full((n,), float("nan"), dtype=torch.float64, device="cuda")
    back = torch.zeros(n, dtype=torch.float64).pin_memory()
    aa.copy(d, h)
    aa.copy(back, d)
    torch.cuda.synchronize()
    assert torch.equal(back, h)
    assert torch.equal(d.cpu(), h)
    # page-locked host and device memory: the kernel path
    L = aa.lib()
    assert L.aa_copy_path(C.c_void_p(d.data_ptr()), C.c_void_p(h.data_ptr())) == 1
    assert L.aa_copy_path(C.c_void_p(back.data_ptr()), C.c_void_p(d.data_ptr())) == 1


@pytest.mark.parametrize("n", [5, 4099])
def test_copy_float32_tail_and_device_to_device(aa, n):
    # 4-byte elements: n * 4 bytes leaves a tail that the 16-byte kernel skips
    h = torch.from_numpy(aa_synth.uniform(6, n).astype(np.float32)).pin_memory()
    d1 = torch.empty(n, dtype=torch.float32, device="cuda")
    d2 = torch.full((n,), float("nan"), dtype=torch.float32, device="cuda")
    aa.copy(d1, h)
    aa.copy(d2, d1)
    torch.cuda.synchronize()
    assert torch.equal(d2.cpu(), h)


def test_copy_pageable_host_falls_back(aa):
    n = 100003
    src = aa_synth.uniform(7, n)  # numpy: pageable host memory
    d = torch.empty(n, dtype=torch.float64, device="cuda")
    rc = aa.lib().aa_copy(C.c_void_p(d.data_ptr()), C.c_void_p(src.ctypes.data), 8 * n,
                          C.c_void_p(torch.cuda.current_stream().cuda_stream))
    torch.cuda.synchronize()
    assert rc == 0
    assert np.array_equal(d.cpu().numpy(), src)
    assert aa.lib().aa_copy_path(C.c_void_p(d.data_ptr()), C.c_void_p(src.ctypes.data)) == 0


def test_copy_rejects_mismatch(aa):
    a = torch.empty(10, dtype=torch.float64, device="cuda")
    with pytest.raises(ValueError):
        aa.copy(a, torch.empty(9, dtype=torch.float64, device="cuda"))
    with pytest.raises(ValueError):
        aa.copy(a, torch.empty(10, dtype=torch.float32, device="cuda"))
