"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle.

FP64 path bar: 1e-10 absolute per amplitude, 1e-9 relative on the norm
fidelity; split factors element by element where pivots are unambiguous.
Mixed path: FP32-class bulk arithmetic, so its bars are stated per test and
derived from FP32 rounding (unit roundoff 6e-8) accumulated over the
contraction lengths involved.
"""

import numpy as np
import pytest

from oracle import mps as omps
from oracle import qr as oqr
from oracle import statevector as sv
from workloads import circuits, gates, states

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__

    __graft_entry__.build()


def gpu_mps(*a, **k):
    from paper_2505_06119_gb300 import MPS

    return MPS(*a, **k)


def sites_statevector(m):
    v = m.get_site(0).reshape(2, -1)
    for i in range(1, m.n):
        s = m.get_site(i)
        v = (v @ s.reshape(s.shape[0], -1)).reshape(-1, s.shape[2])
    return v.reshape(-1)


def placement(cl, cm, cr):
    """Chain length n and site i whose reserved bonds fit (cl, cm, cr) at i, i+1, i+2."""
    e = int(np.ceil(np.log2(max(cl, cm, cr, 2)))) + 1
    return 2 * e + 2, e


def load_two_sites(m, i, a, b):
    """Only sites i, i+1 matter under the local policy; the others keep their
    (unused) initial content."""
    m.set_site(i, a)
    m.set_site(i + 1, b)


def oracle_split(a, b, g, chi):
    """Oracle two-site split of sites a, b under gate g (Sec. III-C.2)."""
    cl, cm, cr = a.shape[0], a.shape[2], b.shape[2]
    x = (a.reshape(2 * cl, cm) @ b.reshape(cm, 2 * cr)).reshape(cl, 2, 2, cr)
    theta = np.einsum("abcd,lcdr->labr", g.reshape(2, 2, 2, 2), x).reshape(2 * cl, 2 * cr)
    q, r, p, disc = oqr.cpqr(theta, kmax=chi)
    right = np.zeros((q.shape[1], 2 * cr), dtype=np.complex128)
    right[:, p] = r
    return q.reshape(cl, 2, -1), right.reshape(-1, 2, cr), disc


SPLIT_CASES = [
    (1, 1, 1, 4),
    (1, 2, 2, 4),
    (2, 3, 5, 3),
    (3, 5, 7, 4),
    (17, 9, 33, 20),
    (40, 40, 40, 40),
    (64, 64, 64, 64),
    (100, 37, 65, 50),
    (130, 70, 129, 128),
    (257, 64, 200, 160),
    # theta at most 64 x 64: the whole split in one CTA (small_gate_kernel)
    (32, 32, 32, 32),
    (32, 32, 32, 20),
    (20, 64, 32, 16),
    (32, 200, 31, 64),
    (5, 4, 30, 64),  # rank of theta = k (with chi_m = 1 the trailing Q columns would be rounding noise)
]


# (cl, cm, cr, chi, max_ctas): max_ctas > 0 caps the panel kernel's grid so that each
# CTA owns more than 128 rows of theta, the regime of chi above ~9700 on the full GPU
SPLIT_CASES_CAPPED = [(257, 64, 200, 160, 2), (300, 80, 300, 300, 1)]


@pytest.mark.parametrize("cl,cm,cr,chi,max_ctas", [c + (0,) for c in SPLIT_CASES] + SPLIT_CASES_CAPPED)
def test_single_split_fp64_matches_oracle(cl, cm, cr, chi, max_ctas):
    """One two-site apply on saturated random sites: new sites equal the oracle's
    Q and R P^T element by element (tie-free Gaussian input, LOCAL policy so no
    centre move is involved)."""
    rng = np.random.default_rng(cl * 7919 + cm * 31 + cr)
    a = states.complex_gaussian(rng, (cl, 2, cm))
    b = states.complex_gaussian(rng, (cm, 2, cr))
    g = gates.haar_unitary(rng, 4)
    n, i = placement(cl, cm, cr)
    chi_cap = max(cl, cm, cr, chi, 4)
    with gpu_mps(n, chi_cap, precision="fp64", policy="local", debug_max_ctas=max_ctas) as m:
        load_two_sites(m, i, a, b)
        m.apply_2q(i, g, chi)
        qa = m.get_site(i)
        rb = m.get_site(i + 1)
        disc, cnt = m.discarded()
    qo, ro, do = oracle_split(a, b, g, chi)
    k = min(2 * cl, 2 * cr, chi)
    assert qa.shape == (cl, 2, k) and rb.shape == (k, 2, cr)
    scale = max(1.0, np.abs(ro).max())
    assert np.abs(qa - qo).max() < 1e-10
    assert np.abs(rb - ro).max() < 1e-10 * scale
    assert cnt == 1
    assert disc == pytest.approx(do, rel=1e-9, abs=1e-12 * scale**2)


@pytest.mark.parametrize("cl,cm,cr,chi", [(3, 5, 7, 4), (40, 40, 40, 40), (130, 70, 129, 128)])
def test_single_split_mixed_close_to_oracle(cl, cm, cr, chi):
    """Mixed path (complex64 data, FP64 norms/pivots): the kept state
    Q R P^T matches the oracle's to ~1e-5 relative (FP32 rounding over
    contractions of length <= 2*max(cl, cr))."""
    rng = np.random.default_rng(cl + 1000 * cr + 17)
    a = states.complex_gaussian(rng, (cl, 2, cm))
    b = states.complex_gaussian(rng, (cm, 2, cr))
    g = gates.haar_unitary(rng, 4)
    n, i = placement(cl, cm, cr)
    with gpu_mps(n, max(cl, cm, cr, chi, 4), precision="mixed", policy="local") as m:
        load_two_sites(m, i, a, b)
        m.apply_2q(i, g, chi)
        qa = m.get_site(i)
        rb = m.get_site(i + 1)
    qo, ro, _ = oracle_split(a, b, g, chi)
    kept_gpu = qa.reshape(2 * cl, -1) @ rb.reshape(rb.shape[0], -1)
    kept_ora = qo.reshape(2 * cl, -1) @ ro.reshape(ro.shape[0], -1)
    rel = np.linalg.norm(kept_gpu - kept_ora) / np.linalg.norm(kept_ora)
    assert rel < 2e-5
    # isometry of the left factor
    q = qa.reshape(2 * cl, -1)
    assert np.abs(q.conj().T @ q - np.eye(q.shape[1])).max() < 1e-5


@pytest.mark.parametrize("policy", ["canon", "local"])
def test_config1_exact_vs_statevector(policy):
    """12-qubit depth-8 Haar brick-wall, complex128, chi_max = 64 (no truncation)."""
    n, depth = 12, 8
    ops = circuits.brickwall(n, depth, seed=1)
    v = sv.run(ops, n)
    with gpu_mps(n, 64, precision="fp64", policy=policy) as m:
        m.run(ops)
        assert abs(m.fidelity() - 1.0) < 1e-9
        rng = np.random.default_rng(2)
        for _ in range(64):
            bits = rng.integers(0, 2, n)
            idx = int("".join(map(str, bits)), 2)
            assert abs(m.amplitude(bits) - v[idx]) < 1e-10
        assert np.abs(sites_statevector(m) - v).max() < 1e-10
        assert max(m.bond_dims()) == 64


@pytest.mark.parametrize("policy", ["canon", "local"])
def test_truncated_circuit_fp64_vs_oracle(policy):
    """Truncation active (chi_max below the exact bond): norm fidelity to 1e-9
    relative and amplitudes to 1e-10 absolute against the oracle, same policy."""
    n, depth, chi = 12, 10, 12
    ops = circuits.brickwall(n, depth, seed=7)
    ref = omps.OracleMPS(n, chi, policy)
    ref.run(ops)
    with gpu_mps(n, chi, precision="fp64", policy=policy) as m:
        m.run(ops)
        assert m.bond_dims() == ref.bond_dims()
        f = m.fidelity()
        assert f == pytest.approx(ref.norm2(), rel=1e-9)
        rng = np.random.default_rng(5)
        for _ in range(64):
            bits = rng.integers(0, 2, n)
            assert abs(m.amplitude(bits) - ref.amplitude(bits)) < 1e-10
        tot, cnt = m.discarded()
        assert cnt == ref.n_two_site
        assert tot == pytest.approx(sum(ref.discarded), rel=1e-8, abs=1e-13)
    assert ref.norm2() < 0.999


def test_truncation_identity_canon_gpu():
    """CANON policy: F = 1 - sum of discarded weights (Sec. III-E), on the GPU."""
    n = 14
    ops = circuits.brickwall(n, 12, seed=21)
    with gpu_mps(n, 16, precision="fp64", policy="canon") as m:
        m.run(ops)
        f = m.fidelity()
        tot, _ = m.discarded()
    assert f < 1.0
    assert f == pytest.approx(1.0 - tot, rel=1e-9)


def test_ghz_and_qft_closed_forms_gpu():
    n = 10
    with gpu_mps(n, 8, precision="fp64") as m:
        m.run(circuits.ghz(n))
        s = 1 / np.sqrt(2)
        assert abs(m.amplitude([0] * n) - s) < 1e-12
        assert abs(m.amplitude([1] * n) - s) < 1e-12
        assert abs(m.amplitude([1] + [0] * (n - 1))) < 1e-12
    t, x = 7, 37
    with gpu_mps(t, 64, precision="fp64") as m:
        m.run(circuits.basis_state(t, x) + circuits.qft_noswap(list(range(t))))
        for y in range(0, 2**t, 5):
            bits = [(y >> (t - 1 - j)) & 1 for j in range(t)]
            rev = sum(b << j for j, b in enumerate(bits))
            want = 2 ** (-t / 2) * np.exp(2j * np.pi * x * rev / 2**t)
            assert abs(m.amplitude(bits) - want) < 1e-12


def test_qpe_dyadic_gpu():
    ops, y = circuits.qpe_dyadic(6, 3, seed=2)
    with gpu_mps(9, 64, precision="fp64") as m:
        m.run(ops)
        v = sites_statevector(m).reshape(2**6, 2**3)
    prob = np.sum(np.abs(v) ** 2, axis=1)
    assert prob[y] == pytest.approx(1.0, abs=1e-10)


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-10), ("mixed", 2e-5)])
def test_routed_grid_circuit_vs_statevector(prec, tol):
    """3x3 grid random circuit (fSim + sqrt gates), vertical couplers routed by SWAP chains."""
    ops = circuits.grid_rcs(3, 3, 6, seed=3)
    v = sv.run(ops, 9)
    with gpu_mps(9, 32, precision=prec) as m:
        m.run(ops)
        assert np.abs(sites_statevector(m) - v).max() < tol


def test_routed_truncated_matches_oracle():
    """Routed grid circuit with truncation.  Haar one-qubit gates keep the column
    norms free of exact ties (the paper's sqrt gates create ties, where two
    correct implementations may pick different pivots)."""
    ops = circuits.grid_rcs(3, 4, 8, seed=11, singles="haar")
    ref = omps.OracleMPS(12, 8, "canon")
    ref.run(ops)
    with gpu_mps(12, 8, precision="fp64") as m:
        m.run(ops)
        assert m.fidelity() == pytest.approx(ref.norm2(), rel=1e-9)
        rng = np.random.default_rng(1)
        for _ in range(32):
            bits = rng.integers(0, 2, 12)
            assert abs(m.amplitude(bits) - ref.amplitude(bits)) < 1e-10


def test_permuted_grid_truncated_matches_oracle():
    """The permutation approach to the vertical couplers (Sec. III-D.2; row snake for
    A/B, column snake for C/D, bubble-sort permutations in between) with truncation:
    norm fidelity, amplitudes and the state against the oracle (Haar 1q gates)."""
    ops = circuits.grid_rcs_permuted(3, 4, 8, seed=11, singles="haar")
    ref = omps.OracleMPS(12, 8, "canon")
    ref.run(ops)
    with gpu_mps(12, 8, precision="fp64") as m:
        m.run(ops)
        assert m.bond_dims() == ref.bond_dims()
        assert m.fidelity() == pytest.approx(ref.norm2(), rel=1e-9)
        rng = np.random.default_rng(2)
        for _ in range(32):
            bits = rng.integers(0, 2, 12)
            assert abs(m.amplitude(bits) - ref.amplitude(bits)) < 1e-10
    assert ref.norm2() < 0.999


def test_centre_moves_keep_state_and_canonical_form():
    n = 10
    ops = circuits.brickwall(n, 6, seed=4)
    v = sv.run(ops, n)
    with gpu_mps(n, 32, precision="fp64", policy="canon") as m:
        m.run(ops)
        for target in (0, 9, 3, 6):
            m.move_centre(target)
            assert m.centre() == target
            assert np.abs(sites_statevector(m) - v).max() < 1e-10
            for i in range(n):
                s = m.get_site(i)
                cl, _, cr = s.shape
                if i < target:
                    a = s.reshape(2 * cl, cr)
                    assert np.abs(a.conj().T @ a - np.eye(cr)).max() < 1e-10
                elif i > target:
                    a = s.reshape(cl, 2 * cr)
                    assert np.abs(a @ a.conj().T - np.eye(cl)).max() < 1e-10
            assert m.fidelity() == pytest.approx(1.0, abs=1e-10)


def test_apply_layer_equals_sequential():
    n, chi = 12, 8
    layers = circuits.brickwall_layers(n, 6, seed=9)
    with gpu_mps(n, chi, precision="fp64", policy="local") as a, gpu_mps(n, chi, precision="fp64", policy="local") as b:
        for ones, twos in layers:
            for q, u in ones:
                a.apply_1q(q, u)
                b.apply_1q(q, u)
            a.apply_layer([q for q, _ in twos], [g for _, g in twos])
            for q, g in twos:
                b.apply_2q(q, g)
        for i in range(n):
            assert np.abs(a.get_site(i) - b.get_site(i)).max() == 0.0


def test_apply_layer_uneven_bonds_matches_one_by_one():
    """A layer over bonds 2..4096 (26 qubits, random canonical state): the gates up to
    chi_l, chi_r = 2048 run concurrently on the layer lanes, the central ones on the
    handle's stream; every site, the bond dims and the discarded weight equal the
    one-by-one result exactly."""
    n, chi = 26, 4096
    sites = states.random_canonical_mps(n, states.max_bond_dims(n, chi), 12, seed=3)
    rng = np.random.default_rng(21)
    bonds = list(range(0, n - 1, 2))
    gs = [gates.haar_unitary(rng, 4) for _ in bonds]
    with gpu_mps(n, chi, precision="mixed", policy="local") as a, gpu_mps(n, chi, precision="mixed", policy="local") as b:
        a.set_sites([x.astype(np.complex64) for x in sites], centre=12)
        b.set_sites([x.astype(np.complex64) for x in sites], centre=12)
        a.apply_layer(bonds, gs)
        for q, g in zip(bonds, gs):
            b.apply_2q(q, g)
        assert a.bond_dims() == b.bond_dims()
        assert a.discarded() == b.discarded()
        for i in range(n):
            assert np.array_equal(a.get_site(i, fmt="c64"), b.get_site(i, fmt="c64")), i


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-10), ("mixed", 2e-5)])
def test_permute_matches_oracle(prec, tol):
    """Site permutation by bubble-sorted SWAPs with truncation (chi = 8 on 9 qubits):
    same SWAP count as the oracle and the same state (Haar gates: no norm ties)."""
    n, chi = 9, 8
    ops = circuits.brickwall(n, 5, seed=17)
    order = list(np.random.default_rng(8).permutation(n))
    o = omps.OracleMPS(n, chi, "canon")
    o.run(ops)
    ns_o = o.permute(order)
    with gpu_mps(n, chi, precision=prec) as m:
        m.run(ops)
        ns = m.permute(order)
        assert ns == ns_o
        assert m.fidelity() == pytest.approx(o.norm2(), rel=1e-9 if prec == "fp64" else 1e-5)
        assert np.abs(sites_statevector(m) - o.statevector()).max() < tol
        with pytest.raises(Exception):
            m.permute([0] * n)


def test_overlap_and_cross_precision():
    n = 10
    ops = circuits.brickwall(n, 6, seed=12)
    v = sv.run(ops, n)
    with gpu_mps(n, 32, precision="fp64") as a, gpu_mps(n, 32, precision="mixed") as b:
        a.run(ops)
        b.run(ops)
        assert a.overlap(a).real == pytest.approx(1.0, abs=1e-10)
        o = a.overlap(b)
        assert abs(o - 1.0) < 1e-5
        assert abs(np.vdot(v, sites_statevector(b)) - o) < 1e-5


def test_get_set_site_roundtrip_and_formats():
    rng = np.random.default_rng(0)
    n = 6
    bonds = states.max_bond_dims(n, 8)
    sites = states.random_canonical_mps(n, bonds, 2, seed=3)
    for prec in ("fp64", "mixed"):
        with gpu_mps(n, 8, precision=prec) as m:
            m.set_sites(sites, centre=2)
            for i in range(n):
                got = m.get_site(i)
                tol = 0 if prec == "fp64" else 1e-7
                assert np.abs(got - sites[i]).max() <= tol
                g64 = m.get_site(i, fmt="c64")
                assert g64.dtype == np.complex64
            assert m.fidelity() == pytest.approx(1.0, abs=1e-6)
    del rng
