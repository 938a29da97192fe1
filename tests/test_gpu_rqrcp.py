"""GPU parity of the randomized-pivoting split (MPS_TRUNC_RQRCP) against its oracle
(oracle/rqrcp.py), through the C ABI.

Both sides draw the same +-1 sketch from SplitMix64 (split number s of a handle uses
the state sketch_seed + s), so in FP64 the pivots agree and the factors are compared
element by element, as for the deterministic pivoted QR.  The mixed path is compared
by the kept state.  Quality: on saturated blocks the randomized pivots discard about
as much weight as QP3's.
"""

import numpy as np
import pytest

from oracle import mps as omps
from oracle import qr as oqr
from oracle import rqrcp as orq
from workloads import circuits, gates, states

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__

    __graft_entry__.build()


def gpu_mps(*a, **k):
    from paper_2505_06119_gb300 import MPS

    return MPS(*a, **k)


def theta_of(a, b, g):
    cl, cm, cr = a.shape[0], a.shape[2], b.shape[2]
    x = (a.reshape(2 * cl, cm) @ b.reshape(cm, 2 * cr)).reshape(cl, 2, 2, cr)
    return np.einsum("abcd,lcdr->labr", np.asarray(g).reshape(2, 2, 2, 2), x).reshape(2 * cl, 2 * cr)


def placement(cl, cm, cr):
    e = int(np.ceil(np.log2(max(cl, cm, cr, 2)))) + 1
    return 2 * e + 2, e


def gpu_split(prec, a, b, g, chi, seed, max_ctas=0):
    cl, cm, cr = a.shape[0], a.shape[2], b.shape[2]
    n, i = placement(cl, cm, cr)
    with gpu_mps(n, max(cl, cm, cr, chi, 4), precision=prec, policy="local", truncation="rqrcp",
                 sketch_seed=seed, debug_max_ctas=max_ctas) as m:
        m.set_site(i, a)
        m.set_site(i + 1, b)
        m.apply_2q(i, g, chi)
        jpvt, k = m.last_pivots()
        qa, rb = m.get_site(i), m.get_site(i + 1)
        disc, _ = m.discarded()
    return qa, rb, jpvt, k, disc


def oracle_split(a, b, g, chi, seed):
    theta = theta_of(a, b, g)
    res = orq.rqrcp(theta, kmax=chi, seed=seed)
    k = res["k"]
    right = np.zeros((k, theta.shape[1]), dtype=np.complex128)
    right[:, res["jpvt"]] = res["r"]
    return theta, res, right


CASES = [(1, 1, 1, 4, 0), (2, 3, 5, 3, 1), (17, 9, 33, 20, 2), (40, 40, 40, 40, 3), (64, 64, 64, 64, 4),
         (100, 37, 65, 50, 5), (130, 70, 129, 128, 6), (257, 64, 200, 160, 7)]


@pytest.mark.parametrize("cl,cm,cr,chi,seed", CASES)
def test_rqrcp_split_fp64_matches_oracle(cl, cm, cr, chi, seed):
    """Same sketch on both sides: the same pivots, Q to 1e-10 and R P^T to 1e-10 of its
    largest entry, the discarded weight to 1e-9 relative (several blocks of 32 pivots,
    ragged last block, tiny shapes)."""
    rng = np.random.default_rng(1000 + 31 * cl + cr)
    a = states.complex_gaussian(rng, (cl, 2, cm))
    b = states.complex_gaussian(rng, (cm, 2, cr))
    g = gates.haar_unitary(rng, 4)
    qa, rb, jpvt, k, disc = gpu_split("fp64", a, b, g, chi, seed)
    theta, res, right = oracle_split(a, b, g, chi, seed)
    assert k == res["k"]
    assert np.array_equal(jpvt[:k], res["jpvt"][:k])
    scale = max(1.0, np.abs(right).max())
    assert np.abs(qa.reshape(2 * cl, k) - res["q"]).max() < 1e-10
    assert np.abs(rb.reshape(k, -1) - right).max() < 1e-10 * scale
    assert disc == pytest.approx(res["discarded"], rel=1e-9, abs=1e-12 * scale**2)


def test_rqrcp_split_fp64_matches_oracle_capped_grid():
    """More than 128 rows per CTA in the panels (the regime of very large bonds)."""
    rng = np.random.default_rng(77)
    a = states.complex_gaussian(rng, (300, 2, 80))
    b = states.complex_gaussian(rng, (80, 2, 300))
    g = gates.haar_unitary(rng, 4)
    qa, rb, jpvt, k, disc = gpu_split("fp64", a, b, g, 300, 9, max_ctas=1)
    theta, res, right = oracle_split(a, b, g, 300, 9)
    assert np.array_equal(jpvt[:k], res["jpvt"][:k])
    assert np.abs(qa.reshape(600, k) - res["q"]).max() < 1e-10
    assert np.abs(rb.reshape(k, -1) - right).max() < 1e-10 * max(1.0, np.abs(right).max())


@pytest.mark.parametrize("chi", [1024])
def test_rqrcp_large_fp64_split_matches_oracle(chi):
    """A saturated bond at chi = 1024 (theta 2048 x 2048, 32 blocks)."""
    rng = np.random.default_rng(5000 + chi)
    a = states.complex_gaussian(rng, (chi, 2, chi)) / np.sqrt(chi)
    b = states.complex_gaussian(rng, (chi, 2, chi)) / np.sqrt(chi)
    g = gates.haar_unitary(rng, 4)
    qa, rb, jpvt, k, disc = gpu_split("fp64", a, b, g, chi, 123)
    theta, res, right = oracle_split(a, b, g, chi, 123)
    assert np.array_equal(jpvt[:k], res["jpvt"][:k])
    assert np.abs(qa.reshape(2 * chi, k) - res["q"]).max() < 1e-10
    assert np.abs(rb.reshape(k, -1) - right).max() < 1e-10 * max(1.0, np.abs(right).max())
    assert disc == pytest.approx(res["discarded"], rel=1e-9)


@pytest.mark.parametrize("cl,cm,cr,chi", [(40, 40, 40, 40), (130, 70, 129, 128)])
def test_rqrcp_split_mixed_close_to_oracle(cl, cm, cr, chi):
    rng = np.random.default_rng(cl + 7 * cr)
    a = states.complex_gaussian(rng, (cl, 2, cm))
    b = states.complex_gaussian(rng, (cm, 2, cr))
    g = gates.haar_unitary(rng, 4)
    qa, rb, jpvt, k, disc = gpu_split("mixed", a, b, g, chi, 4)
    theta, res, right = oracle_split(a, b, g, chi, 4)
    kept_gpu = qa.reshape(2 * cl, k) @ rb.reshape(k, -1)
    kept_ora = res["q"] @ right
    assert np.linalg.norm(kept_gpu - kept_ora) / np.linalg.norm(kept_ora) < 2e-5
    q = qa.reshape(2 * cl, k)
    assert np.abs(q.conj().T @ q - np.eye(k)).max() < 1e-5


@pytest.mark.parametrize("policy", ["canon", "local"])
def test_rqrcp_truncated_circuit_matches_oracle(policy):
    """12-qubit depth-8 Haar brick-wall at chi = 8 with randomized pivots: the state's
    norm fidelity, amplitudes and bond dims equal the oracle's (FP64)."""
    ops = circuits.brickwall(12, 8, seed=31)
    ref = omps.OracleMPS(12, 8, policy, truncation="rqrcp", sketch_seed=42)
    ref.run(ops)
    with gpu_mps(12, 8, precision="fp64", policy=policy, truncation="rqrcp", sketch_seed=42) as m:
        m.run(ops)
        assert m.bond_dims() == ref.bond_dims()
        assert m.fidelity() == pytest.approx(ref.norm2(), rel=1e-9)
        rng = np.random.default_rng(6)
        for _ in range(32):
            bits = rng.integers(0, 2, 12)
            assert abs(m.amplitude(bits) - ref.amplitude(bits)) < 1e-10
        total, cnt = m.discarded()
    assert total == pytest.approx(sum(ref.discarded), rel=1e-8)
    assert ref.norm2() < 0.999


def test_rqrcp_exact_states_and_zero_columns():
    """GHZ and a routed grid circuit without truncation: the randomized split is exact
    (rank-deficient blocks and zero columns included)."""
    from oracle import statevector as sv

    with gpu_mps(10, 16, precision="fp64", truncation="rqrcp") as m:
        m.run(circuits.ghz(10))
        assert abs(m.amplitude([0] * 10) - 2 ** -0.5) < 1e-12
        assert abs(m.amplitude([1] * 10) - 2 ** -0.5) < 1e-12
        assert m.fidelity() == pytest.approx(1.0, abs=1e-12)
    ops = circuits.grid_rcs(3, 3, 6, seed=3)
    v = sv.run(ops, 9)
    for prec, tol in (("fp64", 1e-10), ("mixed", 2e-5)):
        with gpu_mps(9, 32, precision=prec, truncation="rqrcp") as m:
            m.run(ops)
            w = m.get_site(0).reshape(2, -1)
            for i in range(1, 9):
                s = m.get_site(i)
                w = (w @ s.reshape(s.shape[0], -1)).reshape(-1, s.shape[2])
            assert np.abs(w.reshape(-1) - v).max() < tol


@pytest.mark.parametrize("chi", [256, 512])
def test_rqrcp_discards_about_as_much_as_qp3(chi):
    """Saturated Gaussian block (flat spectrum) and a block with a decaying spectrum:
    the randomized pivots' discarded weight is within 10% (flat) and a factor 2
    (decaying) of the deterministic QP3's, both on the GPU (mixed)."""
    rng = np.random.default_rng(chi)
    a = states.complex_gaussian(rng, (chi, 2, chi)) / np.sqrt(chi)
    b = states.complex_gaussian(rng, (chi, 2, chi)) / np.sqrt(chi)
    b *= (0.98 ** np.arange(chi))[None, None, :]  # decaying right bond: a decaying spectrum
    g = gates.haar_unitary(rng, 4)
    n, i = placement(chi, chi, chi)
    out = {}
    for tr in ("qrcp", "rqrcp"):
        with gpu_mps(n, chi, precision="mixed", policy="local", truncation=tr) as m:
            m.set_site(i, a.astype(np.complex64))
            m.set_site(i + 1, b.astype(np.complex64))
            m.apply_2q(i, g, chi // 2)
            out[tr] = m.discarded()[0]
    assert out["qrcp"] > 0
    assert out["rqrcp"] <= 2.0 * out["qrcp"]
    assert out["rqrcp"] >= out["qrcp"] * 0.5
