"""bench.py --impl reference (the CPU oracle's arm) keeps the bench line's
contract on a small workload: one JSON line with the same metric, unit and
direction as the GPU arm, the oracle described in cpu_baseline (OpenMP build
on the host's cores, the whole workload when it fits in host memory), an e2e
object with no host-device traffic, and nothing printed by ranks other than
0."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
ARGS = ["--impl", "reference", "--nx", "40", "--ny", "40", "--nz", "40", "--m", "5",
        "--steps", "2", "--warmup", "1"]


def run(env_extra=None):
    env = dict(os.environ)
    env.update(env_extra or {})
    return subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), *ARGS], cwd=ROOT,
                          env=env, capture_output=True, text=True, timeout=300)


def test_reference_line():
    p = run({"RANK": "0", "WORLD_SIZE": "1"})
    assert p.returncode == 0, p.stderr
    lines = [ln for ln in p.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference"
    assert d["metric"].startswith("AA iterations/s") and "m=5" in d["metric"]
    assert d["unit"] == "iter/s" and d["higher_is_better"] is True
    assert d["steps"] == 2 and d["warmup"] == 1 and d["n_gpus"] == 1
    assert d["value"] > 0 and abs(d["ms_per_step"] - 1e3 / d["value"]) <= 1e-3 * d["ms_per_step"] + 1e-3
    assert d["config"]["n"] == 40 * 40 * 40 and d["config"]["orth"] == "icwy"
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == d["value"]
    # the OpenMP build on every core this process may use (or the reference
    # build on one core where OpenMP is missing)
    assert cb["cores"] in (1, len(os.sched_getaffinity(0)))
    assert "the full workload" in cb["sample"] and "threads" in cb["sample"]
    assert d["config"]["rows_per_step"] == 40 * 40 * 40
    e2e = d["e2e"]
    assert e2e["value"] == d["value"] and e2e["unit"] == "iter/s"
    assert e2e["h2d_bytes_per_step"] == 0 and e2e["d2h_bytes_per_step"] == 0


def test_other_ranks_print_nothing():
    p = run({"RANK": "1", "WORLD_SIZE": "2", "LOCAL_RANK": "1"})
    assert p.returncode == 0, p.stderr
    assert not [ln for ln in p.stdout.splitlines() if ln.startswith("{")]


def test_reference_uses_leading_planes_when_host_memory_is_short(monkeypatch):
    """With too little host memory for the whole problem the reference arm
    runs the leading planes that fit and counts its rate per full-size
    iteration (rows processed / full n)."""
    import argparse
    sys.path.insert(0, ROOT)
    import bench
    args = argparse.Namespace(nx=40, ny=40, nz=40, m=5, orth="icwy", storage="fp64", steps=2,
                              warmup=1)
    per_plane = (2 * 5 + 8) * 40 * 40 * 8
    monkeypatch.setattr(bench, "host_mem_available", lambda: int(10 * per_plane / 0.6))
    d = bench.run_reference(args, 1, 0)
    assert d["config"]["rows_per_step"] == 40 * 40 * 10
    assert "leading 10 of 40 planes" in d["cpu_baseline"]["sample"]
    frac = 10 / 40
    assert abs(d["value"] - 2 * frac / (d["ms_per_step"] * 2e-3)) <= 1e-3 * d["value"]
