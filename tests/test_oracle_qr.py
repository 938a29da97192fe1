"""Pins of the oracle's truncated pivoted Householder QR (CPU only).

The oracle is checked against things it does not share code with: LAPACK's
zgeqp3/zgeqrf (through SciPy/NumPy, same reflector convention), a brute-force
greedy column selection by residual norm, the SVD (Eckart-Young bound) and the
algebraic invariants of a QR with column pivoting (Sec. III-B.2, M = Q R P^T).
"""

import numpy as np
import pytest
import scipy.linalg as sl

from oracle import qr


def cgauss(rng, m, n):
    return (rng.standard_normal((m, n)) + 1j * rng.standard_normal((m, n))) / np.sqrt(2)


SHAPES = [(1, 1), (2, 3), (3, 2), (7, 5), (5, 7), (17, 17), (40, 24), (24, 40), (64, 64), (130, 66)]


@pytest.mark.parametrize("m,n", SHAPES)
def test_matches_lapack_zgeqp3(m, n):
    rng = np.random.default_rng(m * 1000 + n)
    a = cgauss(rng, m, n)
    q, r, p, disc = qr.cpqr(a)
    q2, r2, p2 = sl.qr(a, pivoting=True, mode="economic")
    assert np.array_equal(p, p2)
    scale = np.abs(a).max()
    assert np.abs(r - r2).max() <= 1e-12 * scale * max(m, n)
    assert np.abs(q - q2).max() <= 1e-12 * max(m, n)
    assert disc == 0.0 or disc < 1e-24


@pytest.mark.parametrize("m,n", [(3, 2), (17, 9), (64, 64), (66, 130)])
def test_unpivoted_matches_lapack_zgeqrf(m, n):
    rng = np.random.default_rng(7 + m + n)
    a = cgauss(rng, m, n)
    q, r, p, _ = qr.cpqr(a, pivot=False)
    q2, r2 = np.linalg.qr(a)
    assert np.array_equal(p, np.arange(n))
    assert np.abs(r - r2).max() <= 1e-12 * max(m, n)
    assert np.abs(q - q2).max() <= 1e-12 * max(m, n)


@pytest.mark.parametrize("m,n,k", [(40, 30, 5), (30, 40, 12), (64, 64, 32), (128, 96, 50)])
def test_truncated_is_prefix_of_full(m, n, k):
    """Stopping after k pivots gives the first k steps of the full factorisation."""
    rng = np.random.default_rng(m + 3 * n + k)
    a = cgauss(rng, m, n)
    qf, rf, pf, _ = qr.cpqr(a)
    qt, rt, pt, disc = qr.cpqr(a, kmax=k)
    assert qt.shape == (m, k) and rt.shape == (k, n)
    assert np.array_equal(pt[:k], pf[:k])
    assert np.abs(qt - qf[:, :k]).max() < 1e-12
    assert np.abs(rt[:, :k] - rf[:k, :k]).max() < 1e-12
    # discarded weight = norm^2 of the rows of the full R that are dropped
    assert disc == pytest.approx(np.sum(np.abs(rf[k:, :]) ** 2), rel=1e-11)
    # unitary invariance: ||A||^2 = ||R_k||^2 + discarded
    assert np.sum(np.abs(a) ** 2) == pytest.approx(np.sum(np.abs(rt) ** 2) + disc, rel=1e-12)


@pytest.mark.parametrize("m,n,k", [(20, 20, 20), (33, 17, 10), (17, 33, 17), (50, 50, 25)])
def test_invariants(m, n, k):
    rng = np.random.default_rng(100 + m + n)
    a = cgauss(rng, m, n) @ np.diag(np.logspace(0, -6, n))  # graded columns
    q, r, p, disc = qr.cpqr(a, kmax=k)
    # Q has orthonormal columns
    assert np.abs(q.conj().T @ q - np.eye(q.shape[1])).max() < 1e-13
    # R is upper trapezoidal with a real non-negative... (zlarfg convention: real diagonal)
    assert np.abs(np.tril(r, -1)).max() == 0.0
    assert np.abs(np.diag(r).imag).max() < 1e-14
    # A P = Q R on the kept part when nothing is truncated
    if k == min(m, n):
        assert np.abs(a[:, p] - q @ r).max() < 1e-12
    # |R_jj| nonincreasing and dominating the rest of its row block
    d = np.abs(np.diag(r))
    assert np.all(d[1:] <= d[:-1] * (1 + 1e-12))
    for j in range(r.shape[0]):
        for t in range(j + 1, n):
            assert d[j] ** 2 >= np.sum(np.abs(r[j:, t]) ** 2) * (1 - 1e-12) - 1e-28


def test_pivot_rule_by_brute_force():
    """Each pivot is the column of largest residual norm after projecting out the
    columns already chosen (greedy column selection), lowest index on ties."""
    rng = np.random.default_rng(5)
    m, n, k = 12, 10, 8
    a = cgauss(rng, m, n)
    _, _, p, _ = qr.cpqr(a, kmax=k)
    chosen = []
    for j in range(k):
        if chosen:
            basis, _ = np.linalg.qr(a[:, chosen])
            res = a - basis @ (basis.conj().T @ a)
        else:
            res = a
        norms = np.sum(np.abs(res) ** 2, axis=0)
        norms[chosen] = -1.0
        best = int(np.argmax(norms))
        assert p[j] == best
        chosen.append(best)


@pytest.mark.parametrize("m,n,k", [(16, 16, 4), (32, 20, 10), (20, 32, 10)])
def test_eckart_young_bound(m, n, k):
    """The QR discarded weight can never beat the SVD tail for the same k."""
    rng = np.random.default_rng(m * n + k)
    a = cgauss(rng, m, n)
    _, _, _, disc = qr.cpqr(a, kmax=k)
    s = np.linalg.svd(a, compute_uv=False)
    tail = float(np.sum(s[k:] ** 2))
    assert disc >= tail * (1 - 1e-12)
    assert disc <= float(np.sum(s**2))


def test_zero_and_rank_deficient_columns():
    """Zero columns give tau = 0 (H = I) and no NaN; A P = Q R still holds."""
    rng = np.random.default_rng(11)
    a = cgauss(rng, 8, 6)
    a[:, 1] = 0
    a[:, 4] = 2 * a[:, 0]  # dependent column
    f = qr.factor(a)
    assert np.all(np.isfinite(f["w"])) and np.all(np.isfinite(f["tau"]))
    q = qr.form_q(f)
    r = qr.r_factor(f)
    assert np.abs(a[:, f["jpvt"]] - q @ r).max() < 1e-12
    assert np.abs(q.conj().T @ q - np.eye(6)).max() < 1e-13
    z = np.zeros((5, 4), dtype=np.complex128)
    f = qr.factor(z)
    assert np.all(f["tau"] == 0) and np.array_equal(f["jpvt"], np.arange(4))
    assert np.all(qr.form_q(f) == np.eye(5, 4))


def test_exact_tie_takes_lowest_index():
    a = np.zeros((4, 3), dtype=np.complex128)
    a[0, 0] = 1.0
    a[1, 1] = 2.0
    a[2, 2] = 2.0  # columns 1 and 2 tie exactly
    _, _, p, _ = qr.cpqr(a)
    assert list(p) == [1, 2, 0]


def test_real_reflector_convention():
    """beta = -sign(Re alpha) ||x|| (sign(0) = +1): checked on a 2-vector by hand."""
    a = np.array([[3.0], [4.0]], dtype=np.complex128)
    f = qr.factor(a)
    assert f["w"][0, 0] == pytest.approx(-5.0)
    assert f["tau"][0] == pytest.approx((-5.0 - 3.0) / -5.0)
    assert f["w"][1, 0] == pytest.approx(4.0 / (3.0 + 5.0))
    a = np.array([[-3.0], [4.0]], dtype=np.complex128)
    f = qr.factor(a)
    assert f["w"][0, 0] == pytest.approx(5.0)
    a = np.array([[2j], [0]], dtype=np.complex128)  # complex alpha, zero tail: still reflected
    f = qr.factor(a)
    assert f["w"][0, 0] == pytest.approx(-2.0)
    assert abs(f["tau"][0]) > 0


# ---- pivot-sequence replay (checks of another implementation's pivot choices)

def test_replay_of_own_order_reproduces_factorisation():
    """Replaying the oracle's own pivots gives the same factors bit for bit, and every
    step's chosen norm is the step's largest."""
    rng = np.random.default_rng(41)
    a = cgauss(rng, 50, 37)
    q, r, p, disc = qr.cpqr(a, kmax=20)
    q2, r2, p2, disc2, c2, m2 = qr.cpqr_replay(a, p[:20], kmax=20)
    assert np.array_equal(p, p2)
    assert np.array_equal(q, q2) and np.array_equal(r, r2) and disc == disc2
    assert np.array_equal(c2, m2)


@pytest.mark.parametrize("m,n,k", [(12, 9, 9), (30, 40, 17), (64, 48, 48)])
def test_replay_with_any_order_is_the_qr_of_the_reordered_matrix(m, n, k):
    """With an arbitrary pivot order the replay is the unpivoted Householder QR of the
    chosen columns (LAPACK zgeqrf through NumPy, same reflector convention), R P^T = Q^H A
    on every column, and the per-step norms equal brute-force projections."""
    rng = np.random.default_rng(m + n + k)
    a = cgauss(rng, m, n)
    order = rng.permutation(n)[:k]
    q, r, p, disc, c2, m2 = qr.cpqr_replay(a, order, kmax=k)
    assert np.array_equal(p[:k], order)
    qn, rn = np.linalg.qr(a[:, order])
    assert np.abs(q - qn[:, :k]).max() < 1e-12 * m
    assert np.abs(r[:, :k] - rn[:k, :k]).max() < 1e-12 * m
    assert np.abs(q.conj().T @ a[:, p] - r).max() < 1e-12 * m
    for j in range(k):
        proj = a - qn[:, :j] @ (qn[:, :j].conj().T @ a)
        res = np.sum(np.abs(proj) ** 2, axis=0)
        rest = [t for t in range(n) if t not in set(order[:j].tolist())]
        assert c2[j] == pytest.approx(res[order[j]], rel=1e-10, abs=1e-13)
        assert m2[j] == pytest.approx(res[rest].max(), rel=1e-10, abs=1e-13)
    kept = q @ r
    assert disc == pytest.approx(np.sum(np.abs(a[:, p] - kept) ** 2), rel=1e-10)


def test_replay_flags_a_non_greedy_step():
    rng = np.random.default_rng(43)
    a = cgauss(rng, 20, 16)
    _, _, p, _ = qr.cpqr(a)
    bad = p.copy()
    bad[0], bad[1] = p[1], p[0]  # second-largest norm first
    *_, c2, m2 = qr.cpqr_replay(a, bad)
    assert c2[0] < m2[0]
    with pytest.raises(ValueError):
        qr.cpqr_replay(a, np.zeros(16, dtype=int))  # column 0 twice


def test_column_of_underflowing_residue_gets_the_identity_reflector():
    """A column whose entries' squares underflow (rounding residue around 1e-170 next to
    O(1) columns): the reflector formula would divide by zero; the column is treated as
    zero (tau = 0, R_jj = alpha) and the factorisation stays finite and exact."""
    rng = np.random.default_rng(5)
    a = cgauss(rng, 6, 4)
    a[:, 1] = 0
    a[:, 3] = 1e-170 * (1 + 1j) * cgauss(rng, 6, 1)[:, 0]
    q, r, p, disc = qr.cpqr(a)
    assert np.all(np.isfinite(q)) and np.all(np.isfinite(r))
    assert np.abs(q.conj().T @ q - np.eye(4)).max() < 1e-12
    assert np.abs(q @ r - a[:, p]).max() < 1e-14
    f = qr.factor(a)
    assert f["tau"][3] == 0
