"""CPU oracle for low-synchronization Anderson acceleration (arXiv 2110.09667).

TEST INFRASTRUCTURE ONLY: the test-suite, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg are the only users.  The product path never
imports this package.

Every function here is a thin ctypes marshal over ``aa_oracle.c`` (plain FP64
C, sequential sums, ``-ffp-contract=off``), which follows Algorithms 1-6 of
the paper step by step.  Parity status per function:

- ``qradd`` (MGS, ICWY, CGS-2, DCGS-2), ``qrdelete``, ``lsq``: pinned by the
  uniqueness of the thin QR factorisation (Householder QR), by SVD
  least-squares, by the invariants Q^T Q = I and Q R = F, by the paper's
  synchronization tallies (Sec. 4.1) and by brute-force identities.
- ``step`` / ``solve``: pinned by the Anderson/GMRES equivalence for linear
  maps, the secant identity for n = 1 and finite termination.
- the test-problem maps ``g_*``: pinned by dense-matrix construction and
  closed forms.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "aa_oracle.c")
_LIB_DIR = os.path.join(_HERE, "_build")
_LIB = os.path.join(_LIB_DIR, "liboracle.so")
_LIB_OMP = os.path.join(_LIB_DIR, "liboracle_omp.so")
_lock = threading.Lock()
_libs = {}

MGS, ICWY, CGS2, DCGS2 = 0, 1, 2, 3
ORTH = {"mgs": MGS, "icwy": ICWY, "cgs2": CGS2, "dcgs2": DCGS2}
OK, NOTCONVERGED, BREAKDOWN = 0, 1, 2

_dp = C.POINTER(C.c_double)
GFN = C.CFUNCTYPE(None, _dp, _dp, C.c_int64, C.c_void_p)


class _Problem(C.Structure):
    _fields_ = [("kind", C.c_int), ("nx", C.c_int64), ("ny", C.c_int64), ("nz", C.c_int64),
                ("p0", C.c_double), ("p1", C.c_double), ("p2", C.c_double),
                ("b", _dp), ("fn", GFN), ("user", C.c_void_p)]


def build(force: bool = False, omp: bool = False) -> str:
    """Compile the oracle with gcc: oracle/_build/liboracle.so, the reference
    build (sequential loops and sums), or with omp=True liboracle_omp.so, the
    timed build (the same source with -fopenmp: parallel element-wise loops,
    fixed-chunk dot products combined in chunk order)."""
    out = _LIB_OMP if omp else _LIB
    with _lock:
        if (not force and os.path.exists(out)
                and os.path.getmtime(out) >= os.path.getmtime(_SRC)):
            return out
        os.makedirs(_LIB_DIR, exist_ok=True)
        tmp = out + f".tmp{os.getpid()}"
        flags = ["-fopenmp"] if omp else []
        subprocess.check_call(["gcc", "-O2", "-std=c99", "-fPIC", "-shared", *flags,
                               "-ffp-contract=off", "-fno-fast-math", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, out)
        return out


def set_threads(nthreads: int) -> int:
    """Threads of the timed (OpenMP) build; returns the count in effect."""
    return int(lib(omp=True).ora_set_threads(int(nthreads)))


def lib(omp: bool = False):
    L = _libs.get(omp)
    if L is None:
        L = C.CDLL(build(omp=omp))
        L.ora_create.restype = C.c_void_p
        L.ora_create.argtypes = [C.c_int64, C.c_int, C.c_int]
        L.ora_destroy.argtypes = [C.c_void_p]
        L.ora_set_option.argtypes = [C.c_void_p, C.c_int, C.c_double]
        L.ora_reset.argtypes = [C.c_void_p]
        L.ora_counters.argtypes = [C.c_void_p, C.POINTER(C.c_longlong)]
        L.ora_qradd.argtypes = [C.c_void_p, _dp]
        L.ora_qrdelete.argtypes = [C.c_void_p]
        L.ora_lsq.argtypes = [C.c_void_p, _dp, _dp]
        L.ora_get_qr.argtypes = [C.c_void_p, _dp, _dp, _dp, C.POINTER(C.c_int)]
        L.ora_set_qr.argtypes = [C.c_void_p, _dp, _dp, _dp, C.c_int]
        L.ora_step.argtypes = [C.c_void_p, _dp, _dp, _dp, _dp]
        L.ora_g_jacobi2d.argtypes = [C.c_int64, C.c_int64, C.c_double, _dp, _dp, _dp]
        L.ora_g_jacobi3d.argtypes = [C.c_int64, C.c_int64, C.c_int64, C.c_double, C.c_double,
                                     C.c_double, _dp, _dp, _dp]
        L.ora_g_bratu2d.argtypes = [C.c_int64, C.c_double, _dp, _dp, _dp]
        L.ora_store_round.restype = C.c_double
        L.ora_store_round.argtypes = [C.c_int, C.c_double]
        L.ora_solve.argtypes = [C.c_void_p, C.POINTER(_Problem), _dp, C.c_int, C.c_double,
                                C.c_double, C.c_int, C.c_int, _dp, _dp, C.POINTER(C.c_int)]
        L.ora_set_threads.argtypes = [C.c_int]
        _libs[omp] = L
    return L


def _p(a: np.ndarray | None):
    if a is None:
        return None
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(_dp)


class Oracle:
    """Anderson-acceleration state (Algorithms 1-6) on the CPU, FP64."""

    def __init__(self, n: int, m: int, orth="mgs", *, dcgs2_min_mi: int = 3,
                 dcgs2_scaled: bool = False, store_round: int = 0,
                 breakdown_tol: float = 1e-14, omp: bool = False):
        self.n, self.m = int(n), int(m)
        self.orth = ORTH[orth] if isinstance(orth, str) else int(orth)
        self._L = L = lib(omp)
        self._h = L.ora_create(self.n, self.m, self.orth)
        if not self._h:
            raise MemoryError("ora_create failed")
        L.ora_set_option(self._h, 0, float(dcgs2_min_mi))
        L.ora_set_option(self._h, 1, float(bool(dcgs2_scaled)))
        L.ora_set_option(self._h, 2, float(store_round))
        L.ora_set_option(self._h, 3, float(breakdown_tol))

    def close(self):
        if getattr(self, "_h", None):
            self._L.ora_destroy(self._h)
            self._h = None

    __del__ = close

    def reset(self):
        self._L.ora_reset(self._h)

    def counters(self) -> dict:
        out = (C.c_longlong * 4)()
        self._L.ora_counters(self._h, out)
        return {"syncs_qr": out[0], "syncs_lsq": out[1], "syncs_other": out[2], "cols": out[3]}

    def qradd(self, v: np.ndarray) -> int:
        v = np.ascontiguousarray(v, dtype=np.float64)
        return self._L.ora_qradd(self._h, _p(v))

    def qrdelete(self) -> int:
        return self._L.ora_qrdelete(self._h)

    def lsq(self, f: np.ndarray) -> np.ndarray:
        f = np.ascontiguousarray(f, dtype=np.float64)
        g = np.zeros(self.m, dtype=np.float64)
        k = self._L.ora_lsq(self._h, _p(f), _p(g))
        return g[:k].copy()

    def get_qr(self):
        """Returns (Q n x k, R k x k, T k x k)."""
        Q = np.zeros((self.m, self.n), dtype=np.float64)
        R = np.zeros((self.m, self.m), dtype=np.float64)
        T = np.zeros((self.m, self.m), dtype=np.float64)
        k = C.c_int(0)
        self._L.ora_get_qr(self._h, _p(Q), _p(R), _p(T), C.byref(k))
        k = k.value
        return Q[:k].T.copy(), R[:k, :k].copy(), T[:k, :k].copy()

    def set_qr(self, Q: np.ndarray, R: np.ndarray, T: np.ndarray | None = None):
        k = Q.shape[1]
        Qc = np.ascontiguousarray(Q.T, dtype=np.float64)
        Rf = np.zeros((self.m, self.m))
        Rf[:k, :k] = R
        Tf = None
        if T is not None:
            Tf = np.zeros((self.m, self.m))
            Tf[:k, :k] = T
        self._L.ora_set_qr(self._h, _p(Qc), _p(Rf), _p(Tf), k)

    def step(self, x: np.ndarray, g: np.ndarray):
        """One AA iteration; returns (x_next, ||f_i||, status)."""
        x = np.ascontiguousarray(x, dtype=np.float64)
        g = np.ascontiguousarray(g, dtype=np.float64)
        xn = np.empty(self.n)
        fn = C.c_double(0.0)
        st = self._L.ora_step(self._h, _p(x), _p(g), _p(xn), C.byref(fn))
        return xn, fn.value, st

    def solve(self, problem: dict, x0: np.ndarray, *, max_iters: int, tol: float,
              scale: float = 1.0, stop_kind: int = 0, nrec: int = 0):
        """Algorithm 1 with a built-in map. Returns dict(x, iters, status, resid, rec)."""
        x = np.array(x0, dtype=np.float64, copy=True)
        P, keep = make_problem(problem)
        resid = np.zeros(max_iters + 2)
        rec = np.zeros((max(nrec, 1), self.n))
        it = C.c_int(0)
        st = self._L.ora_solve(self._h, C.byref(P), _p(x), int(max_iters), float(tol),
                             float(scale), int(stop_kind), int(nrec), _p(rec), _p(resid),
                             C.byref(it))
        del keep
        k = it.value
        return {"x": x, "iters": k, "status": st, "resid": resid[: k + 1].copy(),
                "rec": rec[: min(nrec, k)].copy() if nrec else None}


def make_problem(problem: dict):
    """Build the C problem descriptor; returns (struct, objects to keep alive)."""
    kind = problem["kind"]
    P = _Problem()
    keep = []
    null_fn = GFN()
    P.fn = null_fn
    if kind == "jacobi2d":
        b = np.ascontiguousarray(problem["b"], dtype=np.float64)
        keep.append(b)
        P.kind, P.nx, P.ny, P.p0, P.b = 0, problem["nx"], problem["ny"], problem.get("eps", 0.01), _p(b)
    elif kind == "jacobi3d":
        b = np.ascontiguousarray(problem["b"], dtype=np.float64)
        keep.append(b)
        P.kind, P.nx, P.ny, P.nz = 1, problem["nx"], problem["ny"], problem["nz"]
        P.p0, P.p1, P.p2 = problem.get("ey", 0.1), problem.get("ez", 0.01), problem.get("omega", 0.8)
        P.b = _p(b)
    elif kind == "bratu2d":
        src = problem.get("src")
        if src is not None:
            src = np.ascontiguousarray(src, dtype=np.float64)
            keep.append(src)
        P.kind, P.nx, P.p0, P.b = 2, problem["s"], problem["lam"], _p(src)
    elif kind == "callback":
        fn = problem["fn"]

        def _cb(xp, gp, n, user):
            xa = np.ctypeslib.as_array(xp, shape=(n,))
            ga = np.ctypeslib.as_array(gp, shape=(n,))
            ga[:] = fn(xa)

        cb = GFN(_cb)
        keep.append(cb)
        P.kind, P.fn = 3, cb
    else:
        raise ValueError(kind)
    return P, keep


def store_round(mode: int, x: float) -> float:
    """One stored history entry: mode 0 FP64, 1 FP32, 2 BF16 (via FP32)."""
    return lib().ora_store_round(int(mode), float(x))


def g_jacobi2d(nx, ny, eps, b, x):
    gx = np.empty(nx * ny)
    lib().ora_g_jacobi2d(nx, ny, eps, _p(np.ascontiguousarray(b, dtype=np.float64)),
                         _p(np.ascontiguousarray(x, dtype=np.float64)), _p(gx))
    return gx


def g_jacobi3d(nx, ny, nz, ey, ez, omega, b, x, omp: bool = False):
    gx = np.empty(nx * ny * nz)
    lib(omp).ora_g_jacobi3d(nx, ny, nz, ey, ez, omega,
                         _p(np.ascontiguousarray(b, dtype=np.float64)),
                         _p(np.ascontiguousarray(x, dtype=np.float64)), _p(gx))
    return gx


def g_bratu2d(s, lam, src, u):
    gu = np.empty(s * s)
    srcp = None if src is None else np.ascontiguousarray(src, dtype=np.float64)
    lib().ora_g_bratu2d(s, lam, _p(srcp), _p(np.ascontiguousarray(u, dtype=np.float64)), _p(gu))
    return gu
