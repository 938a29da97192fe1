"""Pins of the oracle's MPO zip-up application (CPU only, Sec. III-C.3).

  * the controlled-phase MPO of the IQFT (Sec. III-D.1) as a dense operator is the
    diagonal exp(i c sum_k t_k phi_k) over basis states (closed form);
  * the IQFT with one MPO per control qubit prepares the state of the gate-by-gate
    IQFT, and QPE with it reads out the dyadic phase exactly;
  * zip-up without truncation equals the dense operator on the statevector for random
    MPOs of bond 1 and 2 on random states, both policies, at the chain's ends too, and
    after several MPOs in a row (the recompression of bonds above the chain's bound);
  * with truncation the zip-up keeps left-canonical sites and bonds within chi_max.
"""

import itertools

import numpy as np
import pytest

from oracle import mps as omps
from oracle import statevector as sv
from workloads import circuits, gates, states


def random_mpo(rng, length, bond):
    bonds = [1] + [bond] * (length - 1) + [1]
    return [states.complex_gaussian(rng, (bonds[j], bonds[j + 1], 2, 2)) / 2 for j in range(length)]


def random_state(n, chi, seed, centre=0):
    sites = states.random_canonical_mps(n, states.max_bond_dims(n, chi), centre, seed=seed)
    return sites


def test_controlled_phase_mpo_closed_form():
    phases = [0.3, -1.1, 2.5]
    m = sv.mpo_matrix(circuits.controlled_phase_mpo(phases))
    want = np.zeros(16, dtype=np.complex128)
    for bits in itertools.product([0, 1], repeat=4):
        idx = int("".join(map(str, bits)), 2)
        want[idx] = np.exp(1j * bits[0] * sum(b * p for b, p in zip(bits[1:], phases)))
    assert np.abs(m - np.diag(want)).max() < 1e-15


@pytest.mark.parametrize("t", [2, 3, 6])
def test_iqft_by_mpos_equals_gate_iqft(t):
    n = t + 1
    rng = np.random.default_rng(t)
    v0 = states.complex_gaussian(rng, (2**n,))
    v0 /= np.linalg.norm(v0)
    qs = list(range(1, n))
    a = sv.run(circuits.iqft_mpo(qs), n, v0.copy())
    b = sv.run(circuits.iqft_noswap(qs), n, v0.copy())
    assert np.abs(a - b).max() < 1e-13


@pytest.mark.parametrize("policy", ["canon", "local"])
@pytest.mark.parametrize("first,length,bond", [(0, 7, 2), (1, 5, 2), (2, 2, 2), (3, 4, 1), (0, 3, 2)])
def test_zipup_without_truncation_is_the_dense_operator(policy, first, length, bond):
    n, chi = 7, 64
    rng = np.random.default_rng(first * 10 + length + bond)
    m = omps.OracleMPS(n, chi, policy)
    m.set_sites(random_state(n, chi, seed=length + 3 * first), centre=0)
    v = m.statevector()
    ws = random_mpo(rng, length, bond)
    m.apply_mpo(first, ws)
    want = sv.apply_mpo(v, n, first, ws)
    assert np.abs(m.statevector() - want).max() < 1e-12
    for b, d in enumerate(m.bond_dims()):
        assert d <= omps.physical_bond(n, b, chi)


def test_consecutive_mpos_at_the_edges_stay_exact():
    """Each zip-up may leave a bond above the chain's bound at the ends (the MPO bond
    doubles the carried rank); the recompression brings it back without loss."""
    n, chi = 6, 64
    rng = np.random.default_rng(9)
    m = omps.OracleMPS(n, chi, "canon")
    m.set_sites(random_state(n, chi, seed=4), centre=0)
    v = m.statevector()
    for first, length in [(2, 4), (3, 3), (0, 6), (4, 2)]:
        ws = random_mpo(rng, length, 2)
        m.apply_mpo(first, ws)
        v = sv.apply_mpo(v, n, first, ws)
        assert np.abs(m.statevector() - v).max() < 1e-11
        assert all(d <= omps.physical_bond(n, b, chi) for b, d in enumerate(m.bond_dims()))
    assert max(m.discarded) < 1e-20


def test_qpe_with_iqft_mpos_reads_the_dyadic_phase():
    n_count, n_target = 6, 3
    ops, y = circuits.qpe_dyadic(n_count, n_target, seed=4)
    iq = circuits.iqft_noswap(list(range(n_count)))
    head = ops[: len(ops) - len(iq)]
    mpo_ops = head + circuits.iqft_mpo(list(range(n_count)))
    m = omps.OracleMPS(n_count + n_target, 16, "canon")
    m.run(mpo_ops)
    probs = np.abs(m.statevector().reshape(2**n_count, -1)) ** 2
    assert probs.sum(1)[y] == pytest.approx(1.0, abs=1e-12)


def test_truncated_zipup_keeps_canonical_form():
    n, chi = 10, 8
    m = omps.OracleMPS(n, chi, "canon")
    m.set_sites(random_state(n, chi, seed=2), centre=0)
    f0 = m.norm2()
    discs = m.apply_mpo(1, circuits.controlled_phase_mpo([0.7, -0.4, 1.9, 0.2, -2.2, 1.0, 0.5]))
    assert max(m.bond_dims()) <= chi
    for i in range(m.centre):
        a = m.sites[i].reshape(-1, m.sites[i].shape[2])
        assert np.abs(a.conj().T @ a - np.eye(a.shape[1])).max() < 1e-12
    assert m.norm2() <= f0 * (1 + 1e-12)
    assert len(discs) >= 7 and max(discs) > 0
    # the controlled phases are unitary: without truncation the norm stays
    m2 = omps.OracleMPS(n, 64, "canon")
    m2.set_sites(random_state(n, 64, seed=2), centre=0)
    m2.apply_mpo(1, circuits.controlled_phase_mpo([0.7, -0.4, 1.9, 0.2, -2.2, 1.0, 0.5]))
    assert m2.norm2() == pytest.approx(1.0, abs=1e-12)
