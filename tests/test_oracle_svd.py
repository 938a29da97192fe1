"""Pins of the oracle's truncated-SVD split (CPU only).

The SVD split (Sec. III-B.2 Table III; Schmidt decomposition, Sec. II-A.2) is
checked against what fixes it independently of the LAPACK routine it calls:
  * a matrix built from prescribed singular values and random isometries gives
    those values back, its best rank-k approximation and the Eckart-Young tail;
  * brute force over all unit vectors of C^2 gives the best rank-1 error of a
    2 x 2 block;
  * the Schmidt form cos(a)|00> + e^{ib} sin(a)|11> under local unitaries;
  * no pivoted-QR split of the same rank discards less (Sec. IV-A.1 trade-off);
  * at the MPS level: the statevector without truncation, and under the
    canonical policy F_after = F_before - delta for every split (Sec. III-E).
"""

import numpy as np
import pytest

from oracle import mps as omps
from oracle import qr as oqr
from oracle import statevector as sv
from oracle import svd as osvd
from workloads import circuits, gates, states


def _prescribed(rng, m, n, s0):
    r = len(s0)
    u0 = states.random_isometry(rng, m, r)
    v0 = states.random_isometry(rng, n, r)
    return u0, v0, (u0 * np.asarray(s0)[None, :]) @ v0.conj().T


@pytest.mark.parametrize("m,n", [(12, 10), (10, 12), (16, 16)])
def test_prescribed_spectrum(m, n):
    rng = np.random.default_rng(11)
    s0 = np.array([3.0, 2.5, 2.0, 1.5, 1.0, 0.5, 0.25, 0.1])
    u0, v0, theta = _prescribed(rng, m, n, s0)
    for k in (1, 3, 8, min(m, n)):
        left, right, s, disc = osvd.svd_split(theta, k)
        assert left.shape == (m, k) and right.shape == (k, n)
        assert np.abs(s[:8] - s0).max() < 1e-13
        assert np.abs(s[8:]).max(initial=0.0) < 1e-13
        assert disc == pytest.approx(float(np.sum(s0[k:] ** 2)), abs=1e-13)
        kk = min(k, 8)
        best = (u0[:, :kk] * s0[None, :kk]) @ v0[:, :kk].conj().T
        assert np.abs(left @ right - best).max() < 1e-12
        assert np.abs(left.conj().T @ left - np.eye(k)).max() < 1e-13
        # the kept weight sits in the right site: ||right||^2 + disc = ||theta||^2
        assert np.vdot(right, right).real + disc == pytest.approx(np.vdot(theta, theta).real, rel=1e-13)


def test_rank1_of_2x2_by_brute_force():
    """min over unit x in C^2 of ||theta - x x^H theta||^2 = ||theta||^2 - max ||x^H theta||^2,
    searched on a grid of x = (cos a, e^{ib} sin a)."""
    rng = np.random.default_rng(5)
    for _ in range(3):
        theta = states.complex_gaussian(rng, (2, 2))
        a = np.linspace(0, np.pi / 2, 1501)[:, None]
        b = np.linspace(0, 2 * np.pi, 1501)[None, :]
        x0, x1 = np.cos(a), np.exp(1j * b) * np.sin(a)
        # x^H theta row vector, squared norm, for every grid point
        p = np.abs(np.conj(x0) * theta[0, 0] + np.conj(x1) * theta[1, 0]) ** 2 + \
            np.abs(np.conj(x0) * theta[0, 1] + np.conj(x1) * theta[1, 1]) ** 2
        brute = np.vdot(theta, theta).real - p.max()
        _, _, _, disc = osvd.svd_split(theta, 1)
        assert disc <= brute + 1e-12
        assert disc == pytest.approx(brute, abs=2e-5 * np.vdot(theta, theta).real)


@pytest.mark.parametrize("alpha,beta", [(0.3, 0.0), (0.7, 1.1), (np.pi / 4 - 0.05, 2.0)])
def test_schmidt_closed_form(alpha, beta):
    """cos(a)|00> + e^{ib} sin(a)|11>, then u (x) v: Schmidt coefficients cos a > sin a;
    keeping one leaves cos(a) u|0> (x) v|0> and discards sin^2 a."""
    rng = np.random.default_rng(8)
    u, v = gates.haar_unitary(rng, 2), gates.haar_unitary(rng, 2)
    m = omps.OracleMPS(2, 1, "local", truncation="svd")
    s0 = np.zeros((1, 2, 2), dtype=np.complex128)
    s0[0, 0, 0] = s0[0, 1, 1] = 1.0
    s1 = np.zeros((2, 2, 1), dtype=np.complex128)
    s1[0, 0, 0] = np.cos(alpha)
    s1[1, 1, 0] = np.exp(1j * beta) * np.sin(alpha)
    m.set_sites([s0, s1])
    d = m.apply_2q(0, np.kron(u, v))
    assert d == pytest.approx(np.sin(alpha) ** 2, abs=1e-14)
    assert m.bond_dims() == [1, 1, 1]
    want = np.cos(alpha) * np.kron(u[:, 0], v[:, 0])
    got = m.statevector()
    assert abs(abs(np.vdot(want, got)) - np.cos(alpha) ** 2) < 1e-14
    assert np.vdot(got, got).real == pytest.approx(np.cos(alpha) ** 2, abs=1e-14)


def test_svd_discards_no_more_than_pivoted_qr():
    rng = np.random.default_rng(21)
    for m, n in [(8, 8), (12, 20), (32, 16)]:
        theta = states.complex_gaussian(rng, (m, n))
        for k in (1, 4, min(m, n) // 2, min(m, n) - 1):
            _, _, _, d_svd = osvd.svd_split(theta, k)
            *_, d_qr = oqr.cpqr(theta, kmax=k, pivot=True)
            assert d_svd <= d_qr * (1 + 1e-12) + 1e-15
    # and strictly less on a generic block
    theta = states.complex_gaussian(rng, (16, 16))
    assert osvd.svd_split(theta, 8)[3] < oqr.cpqr(theta, kmax=8, pivot=True)[3]


@pytest.mark.parametrize("policy", ["canon", "local"])
def test_svd_mps_exact_vs_statevector(policy):
    n = 10
    ops = circuits.brickwall(n, 6, seed=3)
    m = omps.OracleMPS(n, 32, policy, truncation="svd")
    m.run(ops)
    assert np.abs(m.statevector() - sv.run(ops, n)).max() < 1e-12
    assert max(m.discarded) < 1e-24


def test_svd_truncation_identity_canon():
    """Canonical policy: every SVD split removes exactly its discarded weight from the
    norm fidelity (Sec. III-E), and the left sites stay isometries."""
    n = 10
    ops = circuits.brickwall(n, 10, seed=6)
    m = omps.OracleMPS(n, 6, "canon", truncation="svd")
    f = 1.0
    for op in ops:
        if op[0] == "1q":
            m.apply_1q(op[1], op[2])
            continue
        d = m.apply_2q(op[1], op[3])
        f_new = m.norm2()
        assert f_new == pytest.approx(f - d, rel=1e-11, abs=1e-14)
        i = op[1]
        a = m.sites[i].reshape(-1, m.sites[i].shape[2])
        assert np.abs(a.conj().T @ a - np.eye(a.shape[1])).max() < 1e-12
        f = f_new
    assert f < 1.0


def test_svd_beats_qr_per_split_and_tracks_overlap():
    """From the same canonical state one SVD split keeps at least the norm a pivoted-QR
    split keeps (Sec. IV-A.1), and the norm fidelity of a truncated SVD run tracks the
    overlap fidelity with the exact state (Sec. III-E), here within 5%."""
    n = 12
    ops = circuits.brickwall(n, 8, seed=4)
    two = [op for op in ops if op[0] != "1q"]
    m_exact = omps.OracleMPS(n, 64, "canon")
    m_exact.run(ops[: len(ops) // 2])
    for op in two[-6:]:
        a, b = m_exact.copy(), m_exact.copy()
        a.truncation = "svd"
        d_svd = a.apply_2q(min(op[1], op[2]), op[3], chi_max=4)
        d_qr = b.apply_2q(min(op[1], op[2]), op[3], chi_max=4)
        assert d_svd <= d_qr * (1 + 1e-12) + 1e-15
    exact = sv.run(ops, n)
    for chi in (12, 20):
        m = omps.OracleMPS(n, chi, "canon", truncation="svd")
        m.run(ops)
        fbar = m.norm2()
        t = m.statevector()
        fov = abs(np.vdot(exact, t)) ** 2 / fbar
        assert 0 < fbar < 1 and 0 < fov < 1
        assert abs(fbar - fov) < 0.05 * fov
