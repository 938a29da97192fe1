"""GPU parity of the MPO zip-up application (mps_apply_mpo, Sec. III-C.3) with the
oracle and the statevector.

Without truncation the zip-up is exact: the state must equal the dense operator
applied to the statevector (FP64 1e-10, mixed 2e-5, the contraction-length bound of
FP32 rounding used elsewhere), for random MPOs of bond 1 and 2, anywhere on the
chain, one after another (which exercises the recompression of bonds above the
chain's bound).  With truncation the splits are pivoted QRs on tie-free blocks, so
the FP64 state, bonds, norm fidelity and discarded weights follow the oracle (1e-9,
1e-10 per amplitude).  The IQFT as controlled-phase MPOs (Sec. III-D.1) is checked on
QPE, whose counting register must end in the dyadic phase.
"""

import numpy as np
import pytest

from oracle import mps as omps
from oracle import statevector as sv
from workloads import circuits, states

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


def random_mpo(rng, length, bond):
    bonds = [1] + [bond] * (length - 1) + [1]
    return [states.complex_gaussian(rng, (bonds[j], bonds[j + 1], 2, 2)) / 2 for j in range(length)]


TOL = {"fp64": 1e-10, "mixed": 2e-5}


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("policy", ["canon", "local"])
def test_zipup_exact_vs_dense_operator(prec, policy):
    n, chi = 8, 64
    rng = np.random.default_rng(17)
    sites = states.random_canonical_mps(n, states.max_bond_dims(n, chi), 0, seed=5)
    ref = omps.OracleMPS(n, chi, policy)
    ref.set_sites(sites, centre=0)
    v = ref.statevector()
    with gpu_mps(n, chi, precision=prec, policy=policy) as m:
        m.set_sites(sites, centre=0)
        for first, length, bond in [(0, 8, 2), (2, 4, 2), (5, 3, 2), (1, 2, 2), (3, 4, 1), (6, 2, 2), (4, 1, 1)]:
            ws = random_mpo(rng, length, bond)
            m.apply_mpo(first, ws)
            ref.apply_mpo(first, ws)
            v = sv.apply_mpo(v, n, first, ws)
            got = sites_statevector(m)
            assert np.abs(got - v).max() < TOL[prec] * max(1.0, np.abs(v).max())
            assert m.bond_dims() == ref.bond_dims()
            assert all(d <= omps.physical_bond(n, b, chi) for b, d in enumerate(m.bond_dims()))


def test_truncated_iqft_mpos_match_oracle():
    """IQFT of 10 qubits as controlled-phase MPOs on a random state of bond 8 at
    chi_max = 8: every zip-up split truncates."""
    n, chi = 10, 8
    sites = states.random_canonical_mps(n, states.max_bond_dims(n, chi), 0, seed=3)
    ops = circuits.iqft_mpo(list(range(n)))
    ref = omps.OracleMPS(n, chi, "canon")
    ref.set_sites(sites, centre=0)
    ref.run(ops)
    with gpu_mps(n, chi, precision="fp64") as m:
        m.set_sites(sites, centre=0)
        m.run(ops)
        assert m.bond_dims() == ref.bond_dims()
        assert m.fidelity() == pytest.approx(ref.norm2(), rel=1e-9)
        assert np.abs(sites_statevector(m) - ref.statevector()).max() < 1e-10
        tot, cnt = m.discarded()
        assert cnt == ref.n_two_site
        assert tot == pytest.approx(sum(ref.discarded), rel=1e-8, abs=1e-14)
    assert ref.norm2() < 0.999


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_qpe_with_iqft_mpos(prec):
    n_count, n_target = 8, 3
    ops, y = circuits.qpe_dyadic(n_count, n_target, seed=6)
    iq = circuits.iqft_noswap(list(range(n_count)))
    ops = ops[: len(ops) - len(iq)] + circuits.iqft_mpo(list(range(n_count)))
    with gpu_mps(n_count + n_target, 16, precision=prec) as m:
        m.run(ops)
        probs = np.abs(sites_statevector(m).reshape(2**n_count, -1)) ** 2
        assert probs.sum(1)[y] == pytest.approx(1.0, abs=1e-5 if prec == "mixed" else 1e-10)


def test_mpo_argument_checks():
    from paper_2505_06119_gb300 import MPSError, _lib as L

    rng = np.random.default_rng(0)
    with gpu_mps(6, 8) as m:
        wide = [states.complex_gaussian(rng, (1, 3, 2, 2)), states.complex_gaussian(rng, (3, 1, 2, 2))]
        with pytest.raises(MPSError) as ei:
            m.apply_mpo(1, wide)
        assert ei.value.code == L.MPS_E_UNSUPPORTED
        with pytest.raises(MPSError) as ei:
            m.apply_mpo(5, random_mpo(rng, 2, 2))  # past the last site
        assert ei.value.code == L.MPS_E_ARG
        bad = [states.complex_gaussian(rng, (2, 2, 2, 2)), states.complex_gaussian(rng, (2, 1, 2, 2))]
        with pytest.raises(MPSError) as ei:
            m.apply_mpo(0, bad)  # first MPO bond must be 1
        assert ei.value.code == L.MPS_E_ARG
