"""Pins of the oracle's truncated QR with randomized column pivoting (CPU only).

The sketching generator is pinned to the published SplitMix64 outputs; the blocked
factorisation is pinned by what does not depend on the oracle's own code: with a
unitary sketch it must choose the pivots of the plain column-pivoted QR (LAPACK
zgeqp3 on tie-free input), the sketch after each block must equal the sketching
matrix times the current residual (computed independently by projection), and the
result must be a QR of the permuted matrix (A P = Q R, Q orthonormal) whose
discarded weight respects the Eckart-Young bound and stays close to the plain
pivoted QR's.
"""

import json
import os

import numpy as np
import pytest
import scipy.linalg as sl

from oracle import qr, rqrcp

HERE = os.path.dirname(os.path.abspath(__file__))


def cgauss(rng, m, n):
    return (rng.standard_normal((m, n)) + 1j * rng.standard_normal((m, n))) / np.sqrt(2)


def test_splitmix64_matches_published_outputs():
    g = json.load(open(os.path.join(HERE, "golden", "splitmix64.json")))
    for case in g["cases"]:
        want = [int(x) for x in case["outputs"]]
        got = rqrcp.splitmix64(np.arange(len(want)), case["seed"])
        assert [int(x) for x in got] == want


def test_sketch_signs_are_balanced_and_seeded():
    a = rqrcp.sketch_signs(40, 1000, seed=5)
    b = rqrcp.sketch_signs(40, 1000, seed=6)
    assert set(np.unique(a.real)) == {-1.0, 1.0} and np.all(a.imag == 0)
    assert abs(a.real.mean()) < 0.02
    assert not np.array_equal(a, b)
    assert np.array_equal(a, rqrcp.sketch_signs(40, 1000, seed=5))


@pytest.mark.parametrize("m,n,k,nb", [(48, 40, 30, 8), (64, 64, 64, 16), (30, 50, 24, 7)])
def test_unitary_sketch_gives_the_plain_pivots(m, n, k, nb):
    """Omega unitary (m x m): the sketch keeps the residual norms, so every block picks
    the pivots of the plain CPQR and the factors agree."""
    rng = np.random.default_rng(m + n + k)
    a = cgauss(rng, m, n)
    om = sl.qr(cgauss(rng, m, m))[0]
    res = rqrcp.rqrcp(a, kmax=k, nb=nb, omega=om)
    q, r, p, d = qr.cpqr(a, kmax=k)
    _, _, p3 = sl.qr(a, pivoting=True, mode="economic")
    assert np.array_equal(res["jpvt"][:k], p[:k]) and np.array_equal(p[:k], p3[:k])
    assert np.abs(res["q"] - q).max() < 1e-11
    assert np.abs(res["r"][:, :k] - r[:, :k]).max() < 1e-11
    assert res["discarded"] == pytest.approx(d, rel=1e-10)


def test_sketch_after_each_block_is_omega_times_the_residual():
    """Duersch-Gu update: after block b the sketch's remaining columns equal
    Omega (I - Q_J Q_J^H) A P restricted to those columns (Q_J from numpy's QR of the
    already chosen columns)."""
    rng = np.random.default_rng(3)
    m, n, k, nb = 60, 50, 40, 10
    a = cgauss(rng, m, n)
    om = rqrcp.sketch_signs(nb + 8, m, seed=11)
    res = rqrcp.rqrcp(a, kmax=k, nb=nb, omega=om, keep_sketches=True)
    assert len(res["sketches"]) == 4
    for b, (y, p) in enumerate(res["sketches"]):
        j1 = min(k, (b + 1) * nb)
        assert np.array_equal(p[:j1], res["jpvt"][:j1])
        qj = np.linalg.qr(a[:, p[:j1]])[0]
        resid = a[:, p] - qj @ (qj.conj().T @ a[:, p])
        assert np.abs(y[:, j1:] - om @ resid[:, j1:]).max() < 1e-10 * np.abs(y).max()


@pytest.mark.parametrize("m,n,k", [(64, 64, 32), (80, 50, 50), (50, 80, 20), (2, 3, 2), (1, 1, 1)])
def test_is_a_truncated_qr_of_the_permuted_matrix(m, n, k):
    rng = np.random.default_rng(7 * m + n)
    a = cgauss(rng, m, n)
    res = rqrcp.rqrcp(a, kmax=k, seed=9)
    q, r, p = res["q"], res["r"], res["jpvt"]
    kk = min(m, n, k)
    assert sorted(p.tolist()) == list(range(n))
    assert np.abs(q.conj().T @ q - np.eye(kk)).max() < 1e-12
    assert np.allclose(np.tril(r, -1), 0)
    assert np.abs(q.conj().T @ a[:, p] - r).max() < 1e-12 * m
    resid = a[:, p] - q @ r
    assert res["discarded"] == pytest.approx(np.sum(np.abs(resid) ** 2), rel=1e-9, abs=1e-20)
    s = np.linalg.svd(a, compute_uv=False)
    assert res["discarded"] >= np.sum(s[kk:] ** 2) * (1 - 1e-12)


def test_discarded_weight_close_to_the_plain_pivoted_qr():
    """Matrices with a decaying spectrum (sigma_i = 2^(-i/8)): the randomized pivots
    keep nearly as much norm as the deterministic ones, block after block (a stale or
    wrong sketch update would lose this after the first block)."""
    rng = np.random.default_rng(21)
    m = n = 256
    u = sl.qr(cgauss(rng, m, m))[0]
    v = sl.qr(cgauss(rng, n, n))[0]
    a = (u * 2.0 ** (-np.arange(m) / 8)) @ v.conj().T
    for k in (32, 64, 128):
        d_qp3 = qr.cpqr(a, kmax=k)[3]
        d_r = rqrcp.rqrcp(a, kmax=k, seed=k)["discarded"]
        tail = np.sum(2.0 ** (-2 * np.arange(k, m) / 8))
        assert tail * (1 - 1e-12) <= d_r <= 4 * d_qp3


def test_rank_deficient_input_has_no_nan():
    """Zero columns and an exactly rank-2 matrix: zero diagonal entries of R11 are
    skipped by the sketch update, the factors stay finite, the discarded weight is 0."""
    rng = np.random.default_rng(4)
    a = cgauss(rng, 20, 2) @ cgauss(rng, 2, 16)
    a[:, 3] = 0
    res = rqrcp.rqrcp(a, kmax=6, nb=4, seed=1)
    assert np.all(np.isfinite(res["q"])) and np.all(np.isfinite(res["r"]))
    assert res["discarded"] < 1e-24
    assert np.abs(res["q"] @ res["r"] - a[:, res["jpvt"]]).max() < 1e-12


def test_mps_with_randomized_pivots_exact_without_truncation_and_norm_identity():
    """As the MPS split: without truncation the state is the statevector's; with it,
    under the canonical policy every split lowers the norm fidelity by its discarded
    weight (Sec. III-E)."""
    from oracle import mps as omps
    from oracle import statevector as sv
    from workloads import circuits

    ops = circuits.brickwall(10, 6, seed=8)
    ref = omps.OracleMPS(10, 32, "canon", truncation="rqrcp", sketch_seed=3)
    ref.run(ops)
    v = ref.sites[0].reshape(2, -1)
    for s in ref.sites[1:]:
        v = (v @ s.reshape(s.shape[0], -1)).reshape(-1, s.shape[2])
    assert np.abs(v.reshape(-1) - sv.run(ops, 10)).max() < 1e-12
    t = omps.OracleMPS(10, 4, "canon", truncation="rqrcp", sketch_seed=3)
    for op in ops:
        if op[0] == "1q":
            t.apply_1q(op[1], op[2])
        else:
            t.move_centre(op[1])
            f0 = t.norm2()
            d = t.apply_2q(op[1], op[3])
            assert t.norm2() == pytest.approx(f0 - d, rel=1e-10, abs=1e-14)
    assert t.norm2() < 0.99
