"""GPU parity of the truncated SVD split (MPS_TRUNC_SVD, one-sided Jacobi) with the
oracle's LAPACK SVD (Sec. III-B.2 Table III; compared with pivoted QR in Sec. IV-A.1).

An SVD split is unique up to a phase per singular vector, so what is unique is
compared: the kept singular values (the row norms of the new right site, in
non-increasing order), the discarded weight, the kept rank-k part left @ right
(unique when sigma_k > sigma_{k+1}; the seeded blocks have gaps), the
Eckart-Young residual ||theta - left @ right||^2 = sum of the discarded squared
singular values (true for any optimal split), and the statevector of an MPS
evolved with SVD splits (each split's phase freedom cancels in it).  The phases
are checked for validity only: the left site is an isometry.

Bars: FP64 1e-10 relative to the block's scale (the Jacobi iteration stops at
|x^H y| <= sqrt(n) eps |x| |y|); mixed 1e-4 (complex64 rotations; a model of the
same iteration in FP32 gives 1e-6 .. 1e-5 at 128 x 128).
"""

import numpy as np
import pytest

from oracle import mps as omps
from oracle import statevector as sv
from oracle import svd as osvd
from workloads import circuits, gates, states

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__

    __graft_entry__.build()


def gpu_mps(*a, **k):
    from paper_2505_06119_gb300 import MPS

    return MPS(*a, **k)


def placement(cl, cm, cr):
    e = int(np.ceil(np.log2(max(cl, cm, cr, 2)))) + 1
    return 2 * e + 2, e


def theta_of(a, b, g):
    cl, cm, cr = a.shape[0], a.shape[2], b.shape[2]
    x = (a.reshape(2 * cl, cm) @ b.reshape(cm, 2 * cr)).reshape(cl, 2, 2, cr)
    return np.einsum("abcd,lcdr->labr", g.reshape(2, 2, 2, 2), x).reshape(2 * cl, 2 * cr)


def sites_statevector(m):
    v = m.get_site(0).reshape(2, -1)
    for i in range(1, m.n):
        s = m.get_site(i)
        v = (v @ s.reshape(s.shape[0], -1)).reshape(-1, s.shape[2])
    return v.reshape(-1)


BARS = {"fp64": 1e-10, "mixed": 1e-4}

# (cl, cm, cr, chi): square, wide and tall blocks, k below and at min(m, n), several
# rounds of 8 warps and a ragged last CTA; cm = 1 gives a rank-4 theta with k = 6
CASES = [
    (1, 1, 1, 4),
    (1, 2, 2, 4),
    (2, 3, 5, 3),
    (3, 5, 7, 4),
    (8, 1, 8, 6),
    (17, 9, 33, 20),
    (40, 40, 40, 40),
    (64, 64, 64, 64),
    (100, 37, 65, 50),
    (130, 70, 129, 128),
]


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("cl,cm,cr,chi", CASES)
def test_single_svd_split_matches_oracle(prec, cl, cm, cr, chi):
    rng = np.random.default_rng(cl * 7919 + cm * 31 + cr + 5)
    a = states.complex_gaussian(rng, (cl, 2, cm))
    b = states.complex_gaussian(rng, (cm, 2, cr))
    g = gates.haar_unitary(rng, 4)
    n, i = placement(cl, cm, cr)
    with gpu_mps(n, max(cl, cm, cr, chi, 4), precision=prec, policy="local", truncation="svd") as m:
        m.set_site(i, a)
        m.set_site(i + 1, b)
        m.apply_2q(i, g, chi)
        left = m.get_site(i).reshape(2 * cl, -1)
        right = m.get_site(i + 1).reshape(-1, 2 * cr)
        disc, cnt = m.discarded()
        assert m.bond_dims()[i + 1] == min(2 * cl, 2 * cr, chi)
    theta = theta_of(a, b, g)
    lo, ro, s, do = osvd.svd_split(theta, chi)
    k = lo.shape[1]
    bar = BARS[prec]
    tot = float(np.vdot(theta, theta).real)
    assert left.shape == (2 * cl, k) and right.shape == (k, 2 * cr) and cnt == 1
    # singular values: row norms of the right site, non-increasing
    sig = np.linalg.norm(right, axis=1)
    assert np.abs(sig - s[:k]).max() < bar * s[0]
    assert disc == pytest.approx(do, abs=bar * tot)
    # left site is an isometry (also where k exceeds the rank of theta)
    assert np.abs(left.conj().T @ left - np.eye(k)).max() < bar * 10
    # Eckart-Young: the residual of the kept part is the discarded weight
    kept = left @ right
    res = float(np.vdot(theta - kept, theta - kept).real)
    assert res == pytest.approx(do, abs=bar * tot)
    # the kept rank-k part itself where it is unique
    if k == len(s) or s[k - 1] - s[k] > 1e-3 * s[0]:
        assert np.abs(kept - lo @ ro).max() < bar * np.abs(theta).max() * 10


@pytest.mark.parametrize("policy", ["canon", "local"])
def test_svd_circuit_fp64_vs_oracle(policy):
    """12-qubit depth-10 brick-wall with SVD truncation at chi_max = 12 (18 truncating
    splits): statevector, norm fidelity and discarded weights against the oracle."""
    n, depth, chi = 12, 10, 12
    ops = circuits.brickwall(n, depth, seed=7)
    ref = omps.OracleMPS(n, chi, policy, truncation="svd")
    ref.run(ops)
    with gpu_mps(n, chi, precision="fp64", policy=policy, truncation="svd") as m:
        m.run(ops)
        assert m.bond_dims() == ref.bond_dims()
        assert m.fidelity() == pytest.approx(ref.norm2(), rel=1e-9)
        assert np.abs(sites_statevector(m) - ref.statevector()).max() < 1e-9
        tot, cnt = m.discarded()
        assert cnt == ref.n_two_site
        assert tot == pytest.approx(sum(ref.discarded), rel=1e-8, abs=1e-13)
    assert ref.norm2() < 0.99


def test_svd_keeps_at_least_the_qr_norm_gpu():
    """Same circuit, both splits on the GPU (CANON): every SVD split discards the least
    a rank-k split can, so the SVD run ends with the larger norm fidelity (Sec. IV-A.1)."""
    n, depth, chi = 12, 10, 12
    ops = circuits.brickwall(n, depth, seed=7)
    f = {}
    for tr in ("qrcp", "svd"):
        with gpu_mps(n, chi, precision="fp64", policy="canon", truncation=tr) as m:
            m.run(ops)
            f[tr] = m.fidelity()
    assert f["svd"] > f["qrcp"]


def test_svd_mixed_circuit_close_to_fp64():
    n, depth, chi = 12, 10, 12
    ops = circuits.brickwall(n, depth, seed=7)
    with gpu_mps(n, chi, precision="fp64", policy="canon", truncation="svd") as a, \
            gpu_mps(n, chi, precision="mixed", policy="canon", truncation="svd") as b:
        a.run(ops)
        b.run(ops)
        fa, fb = a.fidelity(), b.fidelity()
        assert abs(fa - fb) < 1e-5 * fa
        ov = abs(a.overlap(b)) ** 2 / (fa * fb)
        assert 1 - ov < 1e-5


def test_svd_routed_and_layer_paths():
    """SWAP-routed gates and a batched layer use the SVD split too: no truncation
    gives the exact statevector, and a layer equals its gates one by one."""
    n = 8
    rng = np.random.default_rng(2)
    ops = [("2q", 0, 5, gates.haar_unitary(rng, 4)), ("2q", 6, 1, gates.haar_unitary(rng, 4)),
           ("1q", 3, gates.haar_unitary(rng, 2)), ("2q", 2, 7, gates.haar_unitary(rng, 4))]
    with gpu_mps(n, 16, precision="fp64", truncation="svd") as m:
        m.run(ops)
        assert np.abs(sites_statevector(m) - sv.run(ops, n)).max() < 1e-10
    layer = [(q, gates.haar_unitary(rng, 4)) for q in (0, 2, 4, 6)]
    with gpu_mps(n, 4, precision="fp64", policy="local", truncation="svd") as a, \
            gpu_mps(n, 4, precision="fp64", policy="local", truncation="svd") as b:
        for _ in range(2):
            a.apply_layer([q for q, _ in layer], [g for _, g in layer])
            for q, g in layer:
                b.apply_2q(q, g)
            layer = [(q + 1, g) for q, g in layer[:3]]
        assert np.array_equal(sites_statevector(a), sites_statevector(b))
        assert a.discarded() == b.discarded()


def test_svd_bounded_wait_expiry():
    """The Jacobi kernel's grid barrier is bounded like the QR panel's: told to wait
    for one CTA too many it gives up, and the call reports MPS_E_TIMEOUT."""
    from paper_2505_06119_gb300 import MPSError, _lib as L

    m = gpu_mps(6, 8, precision="fp64", policy="local", truncation="svd", wait_timeout_s=0.05,
                debug_barrier_extra=1)
    m.apply_2q(0, gates.haar_unitary(np.random.default_rng(0), 4))
    with pytest.raises(MPSError) as ei:
        m.sync()
    assert ei.value.code == L.MPS_E_TIMEOUT
    m.close()


def test_svd_iteration_record():
    """mps_svd_last_stats reports the sweeps and rotations of the last split; the
    iteration converged (a final sweep without rotations) well inside the limit."""
    from paper_2505_06119_gb300 import MPSError, _lib as L

    rng = np.random.default_rng(3)
    a = states.complex_gaussian(rng, (32, 2, 32))
    b = states.complex_gaussian(rng, (32, 2, 32))
    with gpu_mps(14, 32, precision="mixed", policy="local", truncation="svd") as m:
        assert m.svd_stats() == (0, 0)
        m.set_site(5, a)
        m.set_site(6, b)
        m.apply_2q(5, gates.haar_unitary(rng, 4))
        sweeps, rots = m.svd_stats()
        assert 2 <= sweeps <= 20 and rots >= 64 * 63 // 2
    with gpu_mps(6, 8) as q:
        with pytest.raises(MPSError) as ei:
            q.svd_stats()
        assert ei.value.code == L.MPS_E_STATE
