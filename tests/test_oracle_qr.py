"""Pins for the oracle's QR updates (Algorithms 2-6, QRDelete).

Everything here checks the oracle against facts that do not come from the
oracle itself: uniqueness of the thin QR factorisation (LAPACK Householder
QR through numpy), the invariants Q^T Q = I and Q R = F, the loss-of-
orthogonality orders quoted in Sec. 2.2 / Sec. 3, the synchronization tallies
of Sec. 4.1, and brute-force one-pass CGS for the DCGS-2 start-up identity.
"""
import numpy as np
import pytest

import aa_synth

VARIANTS = ["mgs", "icwy", "cgs2", "dcgs2"]


def householder_qr(F):
    """Thin QR with a positive diagonal (unique for full-rank F)."""
    Q, R = np.linalg.qr(F)
    s = np.sign(np.diag(R))
    s[s == 0] = 1.0
    return Q * s, (R.T * s).T


def build(ora, F, orth, m=None, **kw):
    n, k = F.shape
    O = ora.Oracle(n, m or k, orth, **kw)
    for j in range(k):
        assert O.qradd(F[:, j]) == ora.OK
    return O


@pytest.mark.parametrize("orth", VARIANTS)
def test_qr_matches_householder(ora, orth):
    F = aa_synth.matrix_with_condition(1, 300, 7, 10.0)
    O = build(ora, F, orth)
    Q, R, _ = O.get_qr()
    Qh, Rh = householder_qr(F)
    tol = 1e-12 if orth != "dcgs2" else 1e-10
    assert np.max(np.abs(Q - Qh)) < tol
    assert np.max(np.abs(R - Rh)) / np.max(np.abs(Rh)) < tol
    assert np.linalg.norm(Q @ R - F) / np.linalg.norm(F) < (1e-13 if orth != "dcgs2" else 1e-10)
    assert np.linalg.norm(np.eye(7) - Q.T @ Q) < 1e-12


@pytest.mark.parametrize("orth", VARIANTS)
def test_upper_triangular_positive_diag(ora, orth):
    F = aa_synth.matrix_with_condition(2, 100, 5, 100.0)
    O = build(ora, F, orth)
    _, R, _ = O.get_qr()
    assert np.all(np.diag(R) > 0)
    assert np.allclose(np.tril(R, -1), 0.0, atol=0)


@pytest.mark.parametrize("kappa", [1e4, 1e8])
def test_loss_of_orthogonality_orders(ora, kappa):
    """Sec. 2.2: CGS-2 keeps O(eps) loss; MGS and ICWY O(eps) kappa;
    classical Gram-Schmidt (computed here by brute force) O(eps) kappa^2."""
    F = aa_synth.matrix_with_condition(3, 400, 8, kappa)
    eps = np.finfo(float).eps
    loss = {}
    for orth in VARIANTS:
        Q, _, _ = build(ora, F, orth).get_qr()
        loss[orth] = np.linalg.norm(np.eye(8) - Q.T @ Q)
    # one-pass classical Gram-Schmidt, brute force, for contrast
    Qc = np.zeros_like(F)
    for j in range(8):
        v = F[:, j] - Qc[:, :j] @ (Qc[:, :j].T @ F[:, j])
        Qc[:, j] = v / np.linalg.norm(v)
    loss_cgs = np.linalg.norm(np.eye(8) - Qc.T @ Qc)
    assert loss["cgs2"] < 50 * eps
    assert loss["mgs"] < 50 * eps * kappa
    assert loss["icwy"] < 50 * eps * kappa
    if kappa >= 1e8:
        # MGS is measurably worse than CGS-2 and far better than CGS here.
        assert loss["mgs"] > 10 * loss["cgs2"]
        assert loss_cgs > 100 * loss["mgs"]


def test_icwy_equals_mgs_exact_arithmetic(ora):
    """ICWY is MGS rewritten with a triangular correction (Sec. 3.2); on a
    well-conditioned F they agree to rounding."""
    F = aa_synth.matrix_with_condition(4, 250, 9, 30.0)
    Qm, Rm, _ = build(ora, F, "mgs").get_qr()
    Qi, Ri, Ti = build(ora, F, "icwy").get_qr()
    assert np.max(np.abs(Qm - Qi)) < 1e-13
    assert np.max(np.abs(Rm - Ri)) < 1e-13
    # T = I + L with L_{jl} = q_l^T q_j for the rows computed so far (the last
    # row is the delayed one and still the identity row)
    G = Qi.T @ Qi
    L = np.tril(G, -1)
    L[-1, :] = 0.0
    assert np.max(np.abs(Ti - (np.eye(9) + L))) < 1e-15


def test_dcgs2_startup_is_one_pass_cgs(ora):
    """Algorithm 6 with m_i <= 3 skips the reorthogonalisation, so its first
    three columns are exactly one-pass CGS (brute force here)."""
    F = aa_synth.matrix_with_condition(5, 120, 3, 10.0)
    Q, R, _ = build(ora, F, "dcgs2").get_qr()
    Qc = np.zeros_like(F)
    Rc = np.zeros((3, 3))
    for j in range(3):
        r = Qc[:, :j].T @ F[:, j]
        v = F[:, j] - Qc[:, :j] @ r
        Rc[:j, j] = r
        Rc[j, j] = np.linalg.norm(v)
        Qc[:, j] = v / Rc[j, j]
    assert np.max(np.abs(Q - Qc)) < 1e-14
    assert np.max(np.abs(R - Rc)) < 1e-14


def test_dcgs2_reorth_coefficients(ora):
    """With m_i > 3 DCGS-2 corrects the previous column by the coefficients
    s = Q_{0:k-2}^T q_{k-1} and adds s to R (literal) or R_kk s (scaled)."""
    F = aa_synth.matrix_with_condition(6, 200, 4, 1e6)
    O3 = build(ora, F[:, :3], "dcgs2", m=4)
    Q3, R3, _ = O3.get_qr()
    s = Q3[:, :2].T @ Q3[:, 2]
    for scaled in (False, True):
        O = build(ora, F, "dcgs2", dcgs2_scaled=scaled)
        Q, R, _ = O.get_qr()
        expect = R3[:2, 2] + (R3[2, 2] * s if scaled else s)
        assert np.allclose(R[:2, 2], expect, rtol=0, atol=1e-14 * np.abs(R3).max())
        q2 = Q3[:, 2] - Q3[:, :2] @ s
        assert np.max(np.abs(Q[:, 2] - q2)) < 1e-15


def test_qrdelete_givens(ora):
    """QRDelete: the rotated factors are the (unique) QR of F without its
    first column."""
    F = aa_synth.matrix_with_condition(7, 150, 6, 50.0)
    for orth in VARIANTS:
        O = build(ora, F, orth)
        assert O.qrdelete() == ora.OK
        Q, R, T = O.get_qr()
        assert Q.shape == (150, 5)
        Qh, Rh = householder_qr(F[:, 1:])
        tol = 1e-12 if orth != "dcgs2" else 1e-9
        assert np.max(np.abs(Q - Qh)) < tol
        assert np.max(np.abs(R - Rh)) / np.abs(Rh).max() < tol
        assert np.allclose(np.tril(R, -1), 0.0, atol=0)
        if orth == "icwy":
            # refreshed T: strictly-lower Gram of rotated Q on rows 1..k-2
            G = Q.T @ Q
            L = np.tril(G, -1)
            L[-1, :] = 0.0
            assert np.max(np.abs(T - (np.eye(5) + L))) < 1e-15


@pytest.mark.parametrize("orth,startup,recycle", [
    ("mgs", lambda m: (m * m + m) // 2, lambda m: m),
    ("icwy", lambda m: 2 * m - 1, lambda m: 3),
    ("cgs2", lambda m: 3 * m - 2, lambda m: 3),
    ("dcgs2", lambda m: 2 * m - 1, lambda m: 2),
])
@pytest.mark.parametrize("m", [4, 7])
def test_sync_counts(ora, orth, startup, recycle, m):
    """Sec. 4.1 start-up tallies and the per-iteration recycle counts of
    Sec. 3.1-3.4 (ICWY pays one more reduction to refresh T after a delete)."""
    F = aa_synth.matrix_with_condition(8, 80, m + 3, 10.0)
    O = ora.Oracle(80, m, orth)
    for j in range(m):
        O.qradd(F[:, j])
    assert O.counters()["syncs_qr"] == startup(m)
    for j in range(m, m + 3):
        before = O.counters()["syncs_qr"]
        O.qradd(F[:, j])
        assert O.counters()["syncs_qr"] - before == recycle(m)


@pytest.mark.parametrize("orth", VARIANTS)
def test_breakdown_clears_history(ora, orth):
    F = aa_synth.matrix_with_condition(9, 60, 3, 10.0)
    O = build(ora, F, orth, m=5)
    v = F @ np.array([1.0, -2.0, 0.5])  # in span(Q): rho ~ eps
    assert O.qradd(v) == ora.BREAKDOWN
    assert O.counters()["cols"] == 0
    assert O.qradd(F[:, 0]) == ora.OK


def test_lsq_matches_svd(ora):
    """Algorithm 2: R gamma = Q^T f is the least-squares solution."""
    F = aa_synth.matrix_with_condition(10, 200, 6, 1e3)
    f = aa_synth.uniform(11, 200)
    for orth in VARIANTS:
        O = build(ora, F, orth)
        g = O.lsq(f)
        gs = np.linalg.lstsq(F, f, rcond=None)[0]
        assert np.max(np.abs(g - gs)) <= 1e-10 * np.abs(gs).max()


def test_store_round_fp32(ora):
    """Storage rounding emulation: stored Q entries are exactly fp32 values."""
    F = aa_synth.matrix_with_condition(12, 100, 4, 10.0)
    O = build(ora, F, "cgs2", store_round=1)
    Q, _, _ = O.get_qr()
    assert np.array_equal(Q, Q.astype(np.float32).astype(np.float64))
    assert np.linalg.norm(np.eye(4) - Q.T @ Q) < 1e-6


@pytest.mark.parametrize("orth", ["mgs", "icwy", "cgs2"])
@pytest.mark.parametrize("kappa", [1e6, 1e10])
def test_backward_stability_ill_conditioned(ora, orth, kappa):
    """Gram-Schmidt with correct R columns reproduces F: ||QR - F|| = O(eps)
    ||F|| whatever kappa(F) is.  A dropped reorthogonalisation term in R
    shows up here at the O(eps kappa) level."""
    F = aa_synth.matrix_with_condition(13, 300, 6, kappa)
    Q, R, _ = build(ora, F, orth).get_qr()
    assert np.linalg.norm(Q @ R - F) / np.linalg.norm(F) < 1e-14


@pytest.mark.parametrize("orth", VARIANTS)
def test_new_column_reproduces_v_with_imperfect_Q(ora, orth):
    """For every variant the appended column satisfies v = Q r + rho q_new
    exactly (up to rounding) even when the factor it starts from has lost
    orthogonality (here ~1e-6), because each algorithm subtracts exactly the
    multiples of Q that it records in R.  A coefficient left out of R shows
    up at the 1e-6 level."""
    n, k = 150, 5
    F = aa_synth.matrix_with_condition(14, n, k, 10.0)
    Qh, Rh = householder_qr(F)
    E = aa_synth.uniform(15, n * k).reshape(n, k) * 1e-6
    Qp = Qh + E
    Qp /= np.linalg.norm(Qp, axis=0)
    O = ora.Oracle(n, k + 2, orth, dcgs2_min_mi=99)  # no DCGS-2 reorth of q_{k-1}
    O.set_qr(Qp, Rh, np.eye(k) + np.tril(Qp.T @ Qp, -1))
    v = aa_synth.uniform(16, n)
    assert O.qradd(v) == ora.OK
    Q, R, _ = O.get_qr()
    assert np.linalg.norm(Q @ R[:, k] - v) < 1e-14 * np.linalg.norm(v) * 10
    assert np.max(np.abs(Q[:, :k] - Qp)) == 0.0
