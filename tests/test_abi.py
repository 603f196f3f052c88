"""The C ABI: libaa.so builds for sm_103a, loads on a host without a GPU and
exports every entry point that include/aa.h declares (no compute calls)."""
import ctypes
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for h in os.listdir(os.path.join(ROOT, "include")):
        if not h.endswith(".h"):
            continue
        src = open(os.path.join(ROOT, "include", h)).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_ ]*[\s\*]+(aa_[a-z0-9_]+)\s*\(",
                             src, flags=re.M):
            names.add(m.group(1))
    return names


def test_header_declares_entry_points():
    names = declared_functions()
    for n in ["aa_create", "aa_destroy", "aa_qradd", "aa_lsq", "aa_step", "aa_solve",
              "aa_get_qr", "aa_mdot"]:
        assert n in names


def test_library_exports_every_declared_symbol():
    from paper_2110_09667_gb300 import build
    path = build.build()
    lib = ctypes.CDLL(path)
    missing = [n for n in sorted(declared_functions()) if not hasattr(lib, n)]
    assert not missing, missing


def test_host_only_calls():
    import paper_2110_09667_gb300 as aa
    L = aa.lib()
    assert L.aa_version().startswith(b"libaa")
    assert L.aa_strerror(-4) == b"QR update breakdown (history cleared)"
    cfg = aa.Config()
    L.aa_config_default(ctypes.byref(cfg), 123)
    assert cfg.n == 123 and cfg.m == 5 and cfg.dcgs2_min_mi == 3 and cfg.breakdown_tol == 1e-14
    # argument validation happens before any device call
    h = ctypes.c_void_p()
    cfg.m = 0
    assert L.aa_create(ctypes.byref(cfg), ctypes.byref(h)) == -1
    assert b"m must be" in L.aa_last_error()
