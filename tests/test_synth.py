"""The seeded generators: SplitMix64 known answer and distribution sanity."""
import math

import numpy as np

import aa_synth


def test_splitmix64_known_answer():
    # SplitMix64 seeded with state 0: the first output is 0xE220A8397B1DCDAF
    # (the published generator advances the state by the golden gamma, then mixes).
    z = aa_synth._mix(np.array([0], dtype=np.uint64) + aa_synth.GOLDEN)
    assert int(z[0]) == 0xE220A8397B1DCDAF


def test_uniform_range_and_reproducible():
    a = aa_synth.uniform(3, 100000)
    b = aa_synth.uniform(3, 100000)
    assert np.array_equal(a, b)
    assert a.min() >= -1.0 and a.max() < 1.0
    assert abs(a.mean()) < 0.01 and abs(a.var() - 1.0 / 3.0) < 0.01
    # chunked generation equals one-shot generation
    c = aa_synth.uniform(3, 100000, chunk=777)
    assert np.array_equal(a, c)


def test_normal_moments():
    z = aa_synth.normal(5, 200000)
    assert abs(z.mean()) < 0.01 and abs(z.std() - 1.0) < 0.01


def test_bratu_batch_ranges():
    s, lam = aa_synth.bratu_batch(0, 4096)
    assert s.min() >= 32 and s.max() <= 256
    assert lam.min() >= 1.0 and lam.max() < 6.0
    # log-uniform sides: median near sqrt(32 * 256) = 90.5
    assert 80 <= np.median(s) <= 100


def test_condition_matrix():
    F = aa_synth.matrix_with_condition(0, 200, 6, 1e6)
    sv = np.linalg.svd(F, compute_uv=False)
    assert abs(sv[0] - 1.0) < 1e-12 and abs(sv[-1] / sv[0] - 1e-6) < 1e-12


def test_mixture_samples_moments():
    """The mixture draws have the mixture's mean and variance: mean
    sum a_i mu_i = 0.55, variance sum a_i (s_i^2 + mu_i^2) - mean^2 = 1.1525
    (within 4 standard errors for 10^5 draws), and are reproducible."""
    import numpy as np

    import aa_synth
    x = aa_synth.mixture_samples(3, 100_000)
    assert np.array_equal(x, aa_synth.mixture_samples(3, 100_000))
    mean = 0.3 * 0.0 + 0.3 * 0.5 + 0.4 * 1.0
    var = 0.3 * (1 + 0.0) + 0.3 * (1 + 0.25) + 0.4 * (1 + 1.0) - mean ** 2
    assert abs(x.mean() - mean) < 4 * np.sqrt(var / x.size)
    assert abs(x.var() - var) < 4 * np.sqrt(2 * var ** 2 / x.size) * 1.5


def test_bratu_source_grid_brute_force():
    """f(x_i, y_j) = sum_{k1,k2} c[k1,k2] / (k1^2 + k2^2) sin(k1 pi x_i) sin(k2 pi y_j)
    on the interior grid x_i = i h, h = 1/(s+1), index p = j*s + i, c row-major in
    (k1, k2) (the reading of the source term for the warm-start workload),
    against a direct loop over the points and modes."""
    s, modes = 7, 8
    lam, c = aa_synth.bratu_source_params(3)
    assert 1.0 <= lam <= 6.0 and c.shape == (modes * modes,)
    F = aa_synth.bratu_source_grid(c, s)
    C = np.asarray(c).reshape(modes, modes)
    h = 1.0 / (s + 1)
    for j in range(s):
        for i in range(s):
            ref = sum(C[k1 - 1, k2 - 1] / (k1 * k1 + k2 * k2)
                      * math.sin(k1 * math.pi * (i + 1) * h) * math.sin(k2 * math.pi * (j + 1) * h)
                      for k1 in range(1, modes + 1) for k2 in range(1, modes + 1))
            assert abs(F[j * s + i] - ref) <= 1e-13 * (1 + abs(ref))
    # the first mode alone is a product of sines, symmetric under x <-> y
    e = np.zeros(modes * modes)
    e[0] = 2.0
    F1 = aa_synth.bratu_source_grid(e, s).reshape(s, s)
    assert np.allclose(F1, F1.T, rtol=0, atol=1e-15)
    assert np.all(F1 > 0)


def test_warm_start_features_layout():
    from paper_2110_09667_gb300 import warmstart as ws
    lams = np.array([1.0, 3.5, 6.0])
    cs = np.arange(3 * 64, dtype=np.float64).reshape(3, 64)
    X = ws.features(lams, cs)
    assert X.dtype == np.float32 and X.shape == (3, ws.IN_PAD) and ws.IN_PAD % 8 == 0
    assert np.allclose(X[:, 0], [-5.0 / 3.0, 0.0, 5.0 / 3.0])
    assert np.array_equal(X[:, 1:ws.IN_DIM], cs.astype(np.float32))
    assert not X[:, ws.IN_DIM:].any()
