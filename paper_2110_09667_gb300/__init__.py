"""GB300-native low-synchronization Anderson acceleration (arXiv 2110.09667).

Python binding of libaa (include/aa.h): argument marshalling only.  Every
step of the Anderson iteration runs in the library's sm_103a kernels; this
module passes device pointers (``tensor.data_ptr()``) and the current CUDA
stream.  There is no CPU fallback: importing the binding fails loudly if the
shared library has not been built.
"""
from __future__ import annotations

import ctypes as C  # noqa: N812
import os

from .build import LIB

__all__ = ["Anderson", "Batch", "lib", "mdot", "mdot_noalloc", "AAError", "ORTH", "STORAGE",
           "Jacobi2D", "Jacobi3D", "Bratu2D"]

ORTH = {"mgs": 0, "icwy": 1, "cgs2": 2, "dcgs2": 3}
STORAGE = {"fp64": 0, "fp32": 1, "bf16": 2}
FLAG_DCGS2_SCALED = 0x1
FLAG_ICWY_GRAM = 0x2
FLAG_TIMING = 0x4
FLAG_FP32_DOTS = 0x8
FLAG_DF_ARITH = 0x10
PASS_KINDS = ["init", "A", "proj", "cgs2b", "mgs", "update", "lsq", "mdot"]

AA_OK, AA_NOTCONVERGED = 0, 1
AA_EBREAKDOWN = -4


class AAError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"libaa error {code}: {msg}")
        self.code = code


class Config(C.Structure):
    _fields_ = [("n", C.c_int64), ("m", C.c_int32), ("orth", C.c_int32), ("storage", C.c_int32),
                ("max_iters", C.c_int32), ("tol", C.c_double), ("scale", C.c_double),
                ("stop_kind", C.c_int32), ("dcgs2_min_mi", C.c_int32),
                ("breakdown_tol", C.c_double), ("flags", C.c_uint64), ("stream", C.c_void_p)]


class Stats(C.Structure):
    _fields_ = [("iters", C.c_int64), ("steps", C.c_int64), ("reductions", C.c_int64),
                ("launches", C.c_int64), ("breakdowns", C.c_int64), ("fnorm", C.c_double),
                ("g_ms", C.c_double), ("aa_ms", C.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class Jacobi2D(C.Structure):
    _fields_ = [("nx", C.c_int64), ("ny", C.c_int64), ("eps", C.c_double), ("b_dev", C.c_void_p)]


class Jacobi3D(C.Structure):
    _fields_ = [("nx", C.c_int64), ("ny", C.c_int64), ("nz", C.c_int64), ("ey", C.c_double),
                ("ez", C.c_double), ("omega", C.c_double), ("b_dev", C.c_void_p)]


class Bratu2D(C.Structure):
    _fields_ = [("s", C.c_int64), ("lam", C.c_double), ("src_dev", C.c_void_p)]


GFN = C.CFUNCTYPE(C.c_int, C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p)
_dp = C.POINTER(C.c_double)
_lib = None


def lib():
    """Load libaa.so; raises ImportError if it was not built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB):
            raise ImportError(f"libaa.so not found at {LIB}: run __graft_entry__.build() "
                              "(or python -m paper_2110_09667_gb300.build)")
        L = C.CDLL(LIB)
        L.aa_config_default.argtypes = [C.POINTER(Config), C.c_int64]
        L.aa_create.argtypes = [C.POINTER(Config), C.POINTER(C.c_void_p)]
        L.aa_destroy.argtypes = [C.c_void_p]
        L.aa_reset.argtypes = [C.c_void_p]
        L.aa_set_stream.argtypes = [C.c_void_p, C.c_void_p]
        L.aa_qradd.argtypes = [C.c_void_p, C.c_void_p]
        L.aa_lsq.argtypes = [C.c_void_p, C.c_void_p, _dp]
        L.aa_step.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, _dp]
        L.aa_solve.argtypes = [C.c_void_p, GFN, C.c_void_p, C.c_void_p, C.POINTER(Stats)]
        L.aa_get_qr.argtypes = [C.c_void_p, _dp, _dp, _dp, C.POINTER(C.c_int)]
        L.aa_get_stats.argtypes = [C.c_void_p, C.POINTER(Stats)]
        L.aa_pass_times.argtypes = [C.c_void_p, _dp, C.POINTER(C.c_int64)]
        L.aa_mdot.argtypes = [C.c_void_p, C.c_int64, C.c_int, C.c_void_p, C.c_int64, C.c_int,
                              C.c_int64, _dp, C.c_void_p]
        L.aa_mdot_noalloc.argtypes = [C.c_void_p, C.c_int64, C.c_int, C.c_void_p, C.c_int64,
                                      C.c_int, C.c_int64, C.c_void_p, C.c_void_p]
        L.aa_copy.argtypes = [C.c_void_p, C.c_void_p, C.c_size_t, C.c_void_p]
        L.aa_copy_path.argtypes = [C.c_void_p, C.c_void_p]
        for nm in ("aa_g_jacobi2d", "aa_g_jacobi3d", "aa_g_bratu2d"):
            getattr(L, nm).argtypes = [C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p]
        L.aa_last_error.restype = C.c_char_p
        L.aa_strerror.restype = C.c_char_p
        L.aa_version.restype = C.c_char_p
        _lib = L
    return _lib


def _check(rc: int, allow=(AA_OK,)) -> int:
    if rc in allow:
        return rc
    if rc != AA_OK:
        raise AAError(rc, lib().aa_last_error().decode())
    return rc


def _stream():
    import torch
    return C.c_void_p(torch.cuda.current_stream().cuda_stream)


def _ptr(t) -> C.c_void_p:
    return C.c_void_p(t.data_ptr())


# The C ABI sees only pointers and sizes, so every tensor is checked here
# before its pointer is passed: a wrong dtype, a strided view or a short
# buffer would otherwise make a kernel read or write past its end.  Shapes
# and strides are checked first, then the dtype, then the device.

def _check_dtype_device(*named):
    """(tensor, name) pairs: every dtype first, then every device."""
    import torch
    for t, name in named:
        if t.dtype != torch.float64:
            raise ValueError(f"{name}: expected a float64 tensor, got {t.dtype}")
    for t, name in named:
        if not t.is_cuda:
            raise ValueError(f"{name}: expected a CUDA tensor, got device {t.device}")


def _vec(t, n: int, name: str, dev: bool = True):
    """A float64 CUDA vector holding at least n contiguous values."""
    if t.dim() != 1:
        raise ValueError(f"{name}: expected a 1-D tensor, got shape {tuple(t.shape)}")
    if t.numel() < n:
        raise ValueError(f"{name}: expected at least {n} elements, got {t.numel()}")
    if t.numel() > 1 and t.stride(0) != 1:
        raise ValueError(f"{name}: expected unit stride, got {t.stride(0)}")
    if dev:
        _check_dtype_device((t, name))
    return _ptr(t)


def _cols(t, name: str, n: int | None = None, dev: bool = True):
    """A float64 CUDA matrix whose rows are the columns of the ABI call."""
    if t.dim() != 2:
        raise ValueError(f"{name}: expected a 2-D tensor (columns x n), got shape {tuple(t.shape)}")
    rows, cols = t.shape
    if rows < 1 or cols < 1:
        raise ValueError(f"{name}: empty shape {tuple(t.shape)}")
    if n is not None and cols != n:
        raise ValueError(f"{name}: expected {n} entries per column, got {cols}")
    if cols > 1 and t.stride(1) != 1:
        raise ValueError(f"{name}: entries of a column must be contiguous (stride(1) == 1)")
    if rows > 1 and t.stride(0) < cols:
        raise ValueError(f"{name}: column stride {t.stride(0)} is shorter than n = {cols}")
    if dev:
        _check_dtype_device((t, name))
    return _ptr(t)


def builtin_g(name: str):
    """C function pointer of a built-in map (aa_g_jacobi2d/3d, aa_g_bratu2d)."""
    return GFN(C.cast(getattr(lib(), name), C.c_void_p).value)


class Anderson:
    """One Anderson-acceleration context (aa_create ... aa_destroy)."""

    def __init__(self, n: int, m: int, orth: str = "mgs", storage: str = "fp64", *,
                 tol: float = 1e-8, scale: float = 1.0, max_iters: int = 100,
                 stop_kind: int = 0, dcgs2_min_mi: int = 3, breakdown_tol: float = 1e-14,
                 flags: int = 0, stream=None):
        L = lib()
        cfg = Config()
        L.aa_config_default(C.byref(cfg), int(n))
        cfg.m, cfg.orth, cfg.storage = int(m), ORTH[orth], STORAGE[storage]
        cfg.tol, cfg.scale, cfg.max_iters = float(tol), float(scale), int(max_iters)
        cfg.stop_kind, cfg.dcgs2_min_mi = int(stop_kind), int(dcgs2_min_mi)
        cfg.breakdown_tol, cfg.flags = float(breakdown_tol), int(flags)
        cfg.stream = stream if stream is not None else _stream()
        h = C.c_void_p()
        _check(L.aa_create(C.byref(cfg), C.byref(h)))
        self._h = h
        self.n, self.m = int(n), int(m)
        self.cfg = cfg

    def close(self):
        if getattr(self, "_h", None):
            lib().aa_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_stream(self, stream=None):
        _check(lib().aa_set_stream(self._h, stream if stream is not None else _stream()))

    def reset(self):
        _check(lib().aa_reset(self._h))

    def qradd(self, v) -> int:
        return _check(lib().aa_qradd(self._h, _vec(v, self.n, "v")), allow=(AA_OK, AA_EBREAKDOWN))

    def lsq(self, f):
        import numpy as np
        g = (C.c_double * max(self.m, 1))()
        k = _check(lib().aa_lsq(self._h, _vec(f, self.n, "f"), g), allow=tuple(range(0, self.m + 1)))
        return np.array(g[:k])

    def step(self, x, gx, xnext) -> float:
        fn = C.c_double(0.0)
        _check(lib().aa_step(self._h, _vec(x, self.n, "x"), _vec(gx, self.n, "gx"),
                             _vec(xnext, self.n, "xnext"), C.byref(fn)))
        return fn.value

    def solve(self, gfn, user, x):
        """aa_solve with a C function pointer (builtin_g) and its parameter struct."""
        st = Stats()
        xp = _vec(x, self.n, "x")
        rc = lib().aa_solve(self._h, gfn, C.cast(C.pointer(user), C.c_void_p) if user is not None
                            else None, xp, C.byref(st))
        _check(rc, allow=(AA_OK, AA_NOTCONVERGED))
        return rc, st.as_dict()

    def test_set_device_status(self, code: int):
        """aa_test_set_device_status: plant a device status word (host-side
        fault injection for the error-handling tests)."""
        L = lib()
        L.aa_test_set_device_status.argtypes = [C.c_void_p, C.c_int]
        _check(L.aa_test_set_device_status(self._h, int(code)))

    def get_qr(self):
        import numpy as np
        k = C.c_int(0)
        _check(lib().aa_get_qr(self._h, None, None, None, C.byref(k)))
        k = k.value
        Q = np.zeros((max(k, 1), self.n))
        R = np.zeros((max(k, 1), max(k, 1)))
        T = np.zeros((max(k, 1), max(k, 1)))
        kk = C.c_int(0)
        _check(lib().aa_get_qr(self._h, Q.ctypes.data_as(_dp), R.ctypes.data_as(_dp),
                               T.ctypes.data_as(_dp), C.byref(kk)))
        return Q[:k].T.copy(), R[:k, :k].copy(), T[:k, :k].copy()

    def pass_times(self) -> dict:
        """{kind: (total ms, launches)} from AA_FLAG_TIMING events."""
        ms = (C.c_double * 8)()
        cnt = (C.c_int64 * 8)()
        _check(lib().aa_pass_times(self._h, ms, cnt))
        return {PASS_KINDS[i]: (ms[i], cnt[i]) for i in range(8) if cnt[i]}

    def stats(self) -> dict:
        st = Stats()
        _check(lib().aa_get_stats(self._h, C.byref(st)))
        return st.as_dict()


def mdot(A, V):
    """A^T V for FP64 CUDA tensors A (k x n, rows are columns) and V (nv x n)."""
    import numpy as np
    pa = _cols(A, "A", dev=False)
    k, n = A.shape
    pv = _cols(V, "V", n, dev=False)
    nv = V.shape[0]
    _check_dtype_device((A, "A"), (V, "V"))
    out = np.zeros(k * nv)
    _check(lib().aa_mdot(pa, A.stride(0), k, pv, V.stride(0), nv, n,
                         out.ctypes.data_as(_dp), _stream()))
    return out.reshape(k, nv)


def mdot_noalloc(A, V, out):
    """aa_mdot_noalloc: A^T V into the FP64 CUDA tensor out (k*nv), no allocation."""
    pa = _cols(A, "A", dev=False)
    k, n = A.shape
    pv = _cols(V, "V", n, dev=False)
    nv = V.shape[0]
    po = _vec(out, k * nv, "out", dev=False)
    _check_dtype_device((A, "A"), (V, "V"), (out, "out"))
    rc = lib().aa_mdot_noalloc(pa, A.stride(0), k, pv, V.stride(0), nv, n, po, _stream())
    if rc != AA_OK:
        raise AAError(rc, "aa_mdot_noalloc failed")
    return out


def copy(dst, src):
    """aa_copy: dst <- src (same dtype and element count, contiguous; device
    or page-locked host tensors) on the current stream, by the library's copy
    kernel where the device can address both sides."""
    if dst.dtype != src.dtype:
        raise ValueError(f"copy: dtypes differ ({dst.dtype}, {src.dtype})")
    if dst.numel() != src.numel():
        raise ValueError(f"copy: sizes differ ({dst.numel()}, {src.numel()})")
    if not (dst.is_contiguous() and src.is_contiguous()):
        raise ValueError("copy: tensors must be contiguous")
    for t, name in ((dst, "dst"), (src, "src")):
        if not (t.is_cuda or t.is_pinned()):
            raise ValueError(f"copy: {name} must be a CUDA or page-locked host tensor")
    rc = lib().aa_copy(_ptr(dst), _ptr(src), dst.numel() * dst.element_size(), _stream())
    if rc != AA_OK:
        raise AAError(rc, "aa_copy failed")
    return dst


class BatchDesc(C.Structure):
    _fields_ = [("count", C.c_int32), ("side", C.POINTER(C.c_int64)), ("lam", _dp),
                ("src_host", _dp), ("m", C.c_int32), ("tol", C.c_double),
                ("max_iters", C.c_int32), ("block", C.c_int32), ("ctas_per_sm", C.c_int32)]


def _batch_lib():
    L = lib()
    if not getattr(L, "_batch_ready", False):
        L.aa_batch_create.argtypes = [C.POINTER(BatchDesc), C.POINTER(C.c_void_p)]
        L.aa_batch_destroy.argtypes = [C.c_void_p]
        L.aa_batch_set_x0.argtypes = [C.c_void_p, _dp]
        L.aa_batch_solve.argtypes = [C.c_void_p, C.c_int, C.c_int, C.c_void_p, _dp]
        L.aa_batch_results.argtypes = [C.c_void_p, C.POINTER(C.c_int32), _dp, C.POINTER(C.c_int32)]
        L.aa_batch_solution.argtypes = [C.c_void_p, C.c_int, _dp]
        L.aa_batch_fallbacks.argtypes = [C.c_void_p, C.POINTER(C.c_int32)]
        L.aa_batch_times.argtypes = [C.c_void_p, _dp, _dp]
        L.aa_batch_rows.argtypes = [C.c_void_p]
        L.aa_batch_rows.restype = C.c_int64
        L.aa_batch_set_max_iters.argtypes = [C.c_void_p, C.c_int]
        L.aa_exp_fp32pipe.argtypes = [C.c_int64, C.c_void_p, C.c_void_p, C.c_void_p]
        L._batch_ready = True
    return L


class Batch:
    """Many independent AA(m) Bratu solves in one persistent launch (aa_batch_*)."""

    def __init__(self, sides, lams, *, m: int = 10, tol: float = 1e-8, max_iters: int = 100000,
                 src=None):
        import numpy as np
        L = _batch_lib()
        self.sides = np.ascontiguousarray(sides, dtype=np.int64)
        self.lams = np.ascontiguousarray(lams, dtype=np.float64)
        self.count = len(self.sides)
        self._src = None if src is None else np.ascontiguousarray(src, dtype=np.float64)
        d = BatchDesc()
        d.count = self.count
        d.side = self.sides.ctypes.data_as(C.POINTER(C.c_int64))
        d.lam = self.lams.ctypes.data_as(_dp)
        d.src_host = self._src.ctypes.data_as(_dp) if self._src is not None else None
        d.m, d.tol, d.max_iters = int(m), float(tol), int(max_iters)
        h = C.c_void_p()
        _check(L.aa_batch_create(C.byref(d), C.byref(h)))
        self._h = h

    def close(self):
        if getattr(self, "_h", None):
            _batch_lib().aa_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_x0(self, x0=None):
        import numpy as np
        p = None
        if x0 is not None:
            self._x0 = np.ascontiguousarray(x0, dtype=np.float64)
            p = self._x0.ctypes.data_as(_dp)
        _check(_batch_lib().aa_batch_set_x0(self._h, p))

    def solve(self, block: int = 256, ctas_per_sm: int = 1) -> float:
        ms = C.c_double(0.0)
        _check(_batch_lib().aa_batch_solve(self._h, int(block), int(ctas_per_sm), _stream(),
                                           C.byref(ms)))
        return ms.value

    def results(self):
        import numpy as np
        it = np.zeros(self.count, dtype=np.int32)
        rs = np.zeros(self.count)
        stt = np.zeros(self.count, dtype=np.int32)
        _check(_batch_lib().aa_batch_results(self._h, it.ctypes.data_as(C.POINTER(C.c_int32)),
                                             rs.ctypes.data_as(_dp),
                                             stt.ctypes.data_as(C.POINTER(C.c_int32))))
        return it, rs, stt

    def fallbacks(self):
        import numpy as np
        fb = np.zeros(self.count, dtype=np.int32)
        _check(_batch_lib().aa_batch_fallbacks(self._h, fb.ctypes.data_as(C.POINTER(C.c_int32))))
        return fb

    def times(self):
        """(start_ms, end_ms) per solve of the last solve() call, from the device timer."""
        import numpy as np
        t0 = np.zeros(self.count)
        t1 = np.zeros(self.count)
        _check(_batch_lib().aa_batch_times(self._h, t0.ctypes.data_as(_dp), t1.ctypes.data_as(_dp)))
        return t0, t1

    def solution(self, i: int):
        import numpy as np
        x = np.zeros(int(self.sides[i]) ** 2)
        _check(_batch_lib().aa_batch_solution(self._h, int(i), x.ctypes.data_as(_dp)))
        return x

    def rows(self) -> int:
        return int(_batch_lib().aa_batch_rows(self._h))

    def set_max_iters(self, k: int):
        _check(_batch_lib().aa_batch_set_max_iters(self._h, int(k)))


def exp_fp32pipe(u):
    """e^u on the FP32 pipe (aa_exp_fp32pipe) for an FP64 CUDA tensor."""
    pu = _vec(u, u.numel(), "u")
    out = u.new_empty(u.shape)
    _check(_batch_lib().aa_exp_fp32pipe(u.numel(), pu, _ptr(out), _stream()))
    return out


def selftest_wait_timeout() -> int:
    """aa_selftest_wait_timeout: a device wait that nothing completes must run
    out and come back as AA_ETIMEOUT (the expected return value)."""
    L = lib()
    L.aa_selftest_wait_timeout.argtypes = [C.c_void_p]
    return int(L.aa_selftest_wait_timeout(_stream()))
