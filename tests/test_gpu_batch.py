"""Batched persistent form (many Bratu solves in one launch) against the
oracle: ICWY, m = 10, FP32 history storage (oracle with the same storage
rounding), stop at ||f||/||G(0)|| < 1e-8.

Early iterates are compared with a capped iteration count (both sides
return x_cap); the tolerance follows the precision-form tests (FP32 storage
rounded at slightly different points: 1e-4 relative).  Converged solves must
satisfy the stop rule when checked with the oracle's FP64 map, in an
iteration count within 10 % of the oracle's.
"""
import math

import numpy as np
import pytest

import aa_synth

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

SIDES = [8, 13, 20, 32, 17, 5, 40, 24, 9, 11]


@pytest.fixture(scope="module")
def aa():
    import paper_2110_09667_gb300 as aa
    aa.lib()
    return aa


def scale_of(ora, s, lam, src):
    return float(np.linalg.norm(ora.g_bratu2d(s, lam, src, np.zeros(s * s))))


def oracle_solve(ora, s, lam, src, max_iters, m=10):
    O = ora.Oracle(s * s, m, "icwy", store_round=1)
    sc = scale_of(ora, s, lam, src)
    r = O.solve({"kind": "bratu2d", "s": s, "lam": lam, "src": src}, np.zeros(s * s),
                max_iters=max_iters, tol=1e-8, scale=sc)
    return r, sc


def srcs_for(sides, seed):
    out = []
    for i, s in enumerate(sides):
        out.append(aa_synth.uniform(seed + i, s * s) * 0.5 if i % 2 else np.zeros(s * s))
    return out


def test_batch_early_iterates(aa, ora):
    sides = SIDES
    lams = aa_synth.uniform(70, len(sides), 1.0, 6.0)
    srcs = srcs_for(sides, 71)
    B = aa.Batch(sides, lams, m=10, max_iters=15, src=np.concatenate(srcs))
    B.solve()
    it, rs, st = B.results()
    for i, s in enumerate(sides):
        r, _ = oracle_solve(ora, s, lams[i], srcs[i], 15)
        assert it[i] == r["iters"], (i, it[i], r["iters"])  # 15, or earlier if converged
        xg = B.solution(i)
        assert np.linalg.norm(xg - r["x"]) <= 1e-4 * np.linalg.norm(r["x"]), (i, s)


def test_batch_converges_like_oracle(aa, ora):
    sides = SIDES
    lams = aa_synth.uniform(72, len(sides), 1.0, 6.0)
    srcs = srcs_for(sides, 73)
    B = aa.Batch(sides, lams, m=10, max_iters=20000, src=np.concatenate(srcs))
    B.solve()
    it, rs, st = B.results()
    for i, s in enumerate(sides):
        r, sc = oracle_solve(ora, s, lams[i], srcs[i], 20000)
        assert st[i] == 0 and r["status"] == 0, (i, st[i])
        xg = B.solution(i)
        res = np.linalg.norm(ora.g_bratu2d(s, lams[i], srcs[i], xg) - xg) / sc
        assert res < 1.01e-8, (i, res)
        assert abs(it[i] - r["iters"]) <= max(2, 0.1 * r["iters"]), (i, it[i], r["iters"])


def test_batch_deterministic_and_warm_start(aa, ora):
    sides = [30, 9, 21]
    lams = np.array([2.0, 5.5, 4.0])
    B = aa.Batch(sides, lams, m=10, max_iters=20000)
    B.solve(block=256)
    it0, _, _ = B.results()
    x0 = [B.solution(i) for i in range(3)]
    B.solve(block=256)
    it1, _, _ = B.results()
    assert np.array_equal(it0, it1)
    assert all(np.array_equal(x0[i], B.solution(i)) for i in range(3))
    # warm start: the converged solution needs (almost) no iterations; a
    # wild guess for the second solve falls back to x_0 = 0 and still converges
    guess = [x0[0], np.full(81, 1e3), x0[2]]
    B.set_x0(np.concatenate(guess))
    B.solve(block=128, ctas_per_sm=2)
    it2, rs2, st2 = B.results()
    assert it2[0] <= 1 and it2[2] <= 1 and st2[0] == 0 and st2[2] == 0
    assert st2[1] == 0 and abs(it2[1] - it0[1]) <= max(2, 0.1 * it0[1])


def test_exp_fp32pipe_accuracy(aa):
    """The FP32-pipe exponential used by the batched Bratu map against
    CUDA's FP64 exp (torch.exp on the device).  The (hi, lo) split of u and
    the roundings of the reduced argument's low part err by up to about
    3 |u| 2^-48 absolutely, i.e. relatively in e^u; the polynomial and the
    scaling add a few 2^-48: bound 3 |u| 2^-48 + 2^-45."""
    u = torch.linspace(-20.0, 20.0, 200001, dtype=torch.float64, device="cuda")
    # both sides of every table boundary (multiples of ln2/128 and the odd
    # multiples of ln2/256 where the rounding of u 128/ln2 changes)
    kk = torch.arange(-128 * 120, 128 * 120, dtype=torch.float64, device="cuda")
    step = math.log(2.0) / 256.0
    edges = torch.cat([kk * step * (1 + 1e-12), kk * step * (1 - 1e-12)])
    wide = torch.linspace(-86.0, 86.0, 100001, dtype=torch.float64, device="cuda")
    u = torch.cat([u, edges, wide,
                   torch.tensor([0.0, 1e-30, -1e-30, 0.6931471805599453, 3.0], dtype=torch.float64,
                                device="cuda")])
    got = aa.exp_fp32pipe(u)
    ref = torch.exp(u)
    rel = (got - ref).abs() / ref
    bound = (3.0 * u.abs() + 8.0) * 2.0 ** -48
    assert bool((rel <= bound).all()), (rel / bound).max().item()
    sp = torch.tensor([float("nan"), float("inf"), -float("inf"), 100.0, -100.0], dtype=torch.float64,
                      device="cuda")
    got = aa.exp_fp32pipe(sp).cpu().tolist()
    assert math.isnan(got[0]) and got[1] == math.inf and got[2] == 0.0
    assert got[3] == math.inf and got[4] == 0.0


def test_batch_times_profile(aa):
    """aa_batch_times: every solve has a start no later than its stop, the
    earliest start is 0, and the latest stop lies within the launch's own
    event time; a solve's span grows with its iteration count at a fixed size."""
    sides = [40, 40, 40, 12]
    lams = np.array([2.0, 4.0, 5.5, 3.0])
    B = aa.Batch(sides, lams, m=10, max_iters=20000)
    ms = B.solve(block=256, ctas_per_sm=1)
    it, _, st = B.results()
    t0, t1 = B.times()
    assert np.all(st == 0)
    assert t0.min() == 0.0 and np.all(t1 >= t0)
    assert t1.max() <= ms * 1.05 + 0.05
    same = [0, 1, 2]
    order_it = np.argsort(it[same])
    spans = (t1 - t0)[same]
    assert np.all(np.diff(spans[order_it]) >= -0.02 * spans.max())


def test_batch_full_size_sampled(aa, ora):
    """The 4096-solve workload of the bench (sides log-uniform in [32, 256],
    lambda ~ U(1, 6), zero source) in the bench's launch shape, capped at 3000
    iterations: every solve either meets the stop rule (checked with the
    oracle's FP64 map on 40 converged solves drawn at random) or stops at the
    cap; on 8 capped solves the residual the kernel reports equals the
    oracle's evaluation of the returned iterate."""
    sides, lams = aa_synth.bratu_batch(0, 4096)
    B = aa.Batch(sides, lams, m=10, tol=1e-8, max_iters=3000)
    B.solve(512, 1)
    it, rs, st = B.results()
    assert set(np.unique(st)) <= {0, 1}
    assert np.all(it[st == 1] == 3000) and np.all(it[st == 0] <= 3000)
    rng = np.random.default_rng(5)
    conv = np.flatnonzero(st == 0)
    capped = np.flatnonzero(st == 1)
    assert conv.size > 1000 and capped.size > 100
    for i in rng.choice(conv, 40, replace=False):
        s, lam = int(sides[i]), float(lams[i])
        x = B.solution(int(i))
        sc = scale_of(ora, s, lam, None)
        res = np.linalg.norm(ora.g_bratu2d(s, lam, None, x) - x) / sc
        assert res < 1.01e-8, (i, s, lam, res)
    for i in rng.choice(capped, 8, replace=False):
        s, lam = int(sides[i]), float(lams[i])
        x = B.solution(int(i))
        sc = scale_of(ora, s, lam, None)
        res = np.linalg.norm(ora.g_bratu2d(s, lam, None, x) - x) / sc
        # the kernel reports ||f|| of the returned iterate
        assert abs(res - rs[i]) <= 1e-6 * res + 1e-14, (i, res, rs[i])
        assert res >= 1e-8


def test_batch_early_iterates_large_sides(aa, ora):
    """Early iterates at the workload's large sides: a 256 x 256 solve streams
    128 row blocks of 512 rows through each CTA's cp.async double buffer
    (a 128 x 128 solve 32), so the buffer's refill and wait order is
    compared with the oracle, not only its first blocks."""
    sides = [256, 128, 200, 97]
    lams = np.array([1.5, 5.0, 3.0, 6.0])
    srcs = srcs_for(sides, 74)
    B = aa.Batch(sides, lams, m=10, max_iters=15, src=np.concatenate(srcs))
    B.solve(block=512)
    it, rs, st = B.results()
    for i, s in enumerate(sides):
        r, _ = oracle_solve(ora, s, lams[i], srcs[i], 15)
        assert it[i] == r["iters"], (i, it[i], r["iters"])
        xg = B.solution(i)
        d = xg - r["x"]
        assert np.linalg.norm(d) <= 1e-4 * np.linalg.norm(r["x"]), (i, s)
        assert np.max(np.abs(d)) <= 1e-4 * np.max(np.abs(r["x"])), (i, s)
