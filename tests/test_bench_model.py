"""The roofline model of bench.py: algorithmic bytes and FP64 flops per row
of each pass at a full history, against the counts written out by hand from
the passes' reads, writes and multiply-adds (ICWY, m = 20, FP64: pass A
reads x, G(x), G(x_prev), f_prev and 20 history columns, writes dG, df, f,
G(x) and 19 rotated columns = 376 bytes; 19 rotations x 2 multiply-adds,
3 differences, 59 dot-product terms x 2 = 197 flops)."""
import importlib.util
import os

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def bench():
    spec = importlib.util.spec_from_file_location("bench_mod", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_pass_a_icwy_m20():
    b = bench()
    assert b.pass_bytes("A", 1, 20, 8, "icwy") == 4 * 8 + 20 * 8 + 8 + 3 * 8 + 19 * 8 == 376
    assert b.pass_flops("A", 1, 20, "icwy") == 19 * 4 + 3 + 2 * (3 + 19 + 19 + 18) == 197


def test_other_passes_and_storage():
    b = bench()
    # projection: read df, f and 19 columns, write the new column
    assert b.pass_bytes("proj", 1, 20, 8, "icwy") == 2 * 8 + 19 * 8 + 8 == 176
    # update: read G(x) and 20 dG columns, write x
    assert b.pass_bytes("update", 1, 20, 8, "icwy") == 8 + 20 * 8 + 8 == 176
    assert b.pass_flops("update", 1, 20, "icwy") == 40
    # FP32 history halves only the history terms
    assert b.pass_bytes("A", 1, 20, 4, "icwy") == 4 * 8 + 20 * 4 + 4 + 3 * 8 + 19 * 4 == 216
    # MGS link: read v and two columns, write v
    assert b.pass_bytes("mgs", 1, 20, 8, "mgs") == 32


def test_peaks():
    b = bench()
    assert abs(b.FP64_PEAK_TFLOPS - 2 * 2 * 152 * 2.07e9 / 1e12) < 1e-12
