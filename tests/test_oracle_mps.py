"""Pins of the oracle's MPS evolution (CPU only).

Checked against the brute-force statevector (no truncation), closed forms
(Bell/GHZ, QFT of a basis state, phase estimation), the paper's printed gates
and state examples (tests/golden), and the truncation identities of the
norm fidelity (Sec. III-E).
"""

import json
import os

import numpy as np
import pytest

from oracle import mps as omps
from oracle import statevector as sv
from workloads import circuits, gates, states

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def load(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return json.load(f)


def cmat(rows):
    return np.array([[complex(re, im) for re, im in row] for row in rows])


def test_gate_fixtures_match_paper():
    g = load("paper_gates.json")
    s = 1 / np.sqrt(2)
    for name, fn in [("hadamard", gates.hadamard), ("sqrt_x", gates.sqrt_x),
                     ("sqrt_y", gates.sqrt_y), ("sqrt_w", gates.sqrt_w), ("fsim", gates.fsim)]:
        m = cmat(g[name]["m"]) * (s if g[name]["scale"] == "s" else 1.0)
        assert np.abs(fn() - m).max() < 1e-15, name
        assert np.abs(fn().conj().T @ fn() - np.eye(len(m))).max() < 1e-14
    assert np.abs(gates.r_k(2) - cmat(g["r_k"]["k2"])).max() < 1e-15
    assert np.abs(gates.r_k(3) - cmat(g["r_k"]["k3"])).max() < 1e-15


def test_bell_state_golden():
    b = load("bell_state.json")
    m = omps.OracleMPS(2, 4)
    m.run(circuits.ghz(2))
    ref = np.array([complex(*x) for x in b["amplitudes"]])
    assert np.abs(m.statevector() - ref).max() < 1e-15


def test_tensor_product_order_golden():
    p = load("tensor_product_order.json")
    a1, b1 = [complex(*x) for x in p["psi1"]]
    a2, b2 = [complex(*x) for x in p["psi2"]]

    def prep(a, b):  # unitary with first column (a, b)
        return np.array([[a, -np.conj(b)], [b, np.conj(a)]])

    m = omps.OracleMPS(2, 4)
    m.apply_1q(0, prep(a1, b1))
    m.apply_1q(1, prep(a2, b2))
    want = {"a1a2": a1 * a2, "a1b2": a1 * b2, "b1a2": b1 * a2, "b1b2": b1 * b2}
    for idx, key in enumerate(p["order"]):
        bits = [(idx >> 1) & 1, idx & 1]
        assert m.amplitude(bits) == pytest.approx(want[key], abs=1e-15)


@pytest.mark.parametrize("policy", ["canon", "local"])
def test_brickwall_exact_vs_statevector(policy):
    """12-qubit depth-8 Haar brick-wall, chi_max = 64: no truncation, F = 1."""
    n, depth = 12, 8
    ops = circuits.brickwall(n, depth, seed=1)
    m = omps.OracleMPS(n, 64, policy)
    m.run(ops)
    v = sv.run(ops, n)
    assert np.abs(m.statevector() - v).max() < 1e-12
    assert m.norm2() == pytest.approx(1.0, abs=1e-12)
    assert max(m.bond_dims()) == 64
    rng = np.random.default_rng(3)
    for _ in range(20):
        bits = rng.integers(0, 2, n)
        idx = int("".join(map(str, bits)), 2)
        assert abs(m.amplitude(bits) - v[idx]) < 1e-12
    assert max(m.discarded) < 1e-24


@pytest.mark.parametrize("n", [2, 5, 9])
def test_ghz_closed_form(n):
    m = omps.OracleMPS(n, 8)
    m.run(circuits.ghz(n))
    s = 1 / np.sqrt(2)
    assert m.amplitude([0] * n) == pytest.approx(s, abs=1e-14)
    assert m.amplitude([1] * n) == pytest.approx(s, abs=1e-14)
    v = m.statevector()
    v[0] -= s
    v[-1] -= s
    assert np.abs(v).max() < 1e-14


@pytest.mark.parametrize("x", [0, 5, 37])
def test_qft_of_basis_state_closed_form(x):
    """QFT (swaps omitted) of |x>: amplitude of |y> is 2^{-t/2} exp(2 pi i x rev(y) / 2^t),
    rev(y) = sum_j y_j 2^j with y_j the bit on position j."""
    t = 7
    ops = circuits.basis_state(t, x) + circuits.qft_noswap(list(range(t)))
    m = omps.OracleMPS(t, 64)
    m.run(ops)
    v = m.statevector()
    for y in range(2**t):
        bits = [(y >> (t - 1 - j)) & 1 for j in range(t)]
        rev = sum(b << j for j, b in enumerate(bits))
        want = 2 ** (-t / 2) * np.exp(2j * np.pi * x * rev / 2**t)
        assert abs(v[y] - want) < 1e-13


def test_iqft_inverts_qft():
    t = 6
    rng = np.random.default_rng(4)
    ops = circuits.brickwall(t, 3, seed=9)
    ref = sv.run(ops, t)
    m = omps.OracleMPS(t, 64)
    m.run(ops + circuits.qft_noswap(list(range(t))) + circuits.iqft_noswap(list(range(t))))
    assert np.abs(m.statevector() - ref).max() < 1e-12
    del rng


def test_qpe_dyadic_exact():
    ops, y = circuits.qpe_dyadic(6, 3, seed=2)
    m = omps.OracleMPS(9, 64)
    m.run(ops)
    v = m.statevector().reshape(2**6, 2**3)
    prob = np.sum(np.abs(v) ** 2, axis=1)
    assert prob[y] == pytest.approx(1.0, abs=1e-12)


def test_qpe_fejer_kernel():
    tc, tt = 6, 3
    ops, phi = circuits.qpe(tc, tt, seed=5)
    m = omps.OracleMPS(tc + tt, 64)
    m.run(ops)
    v = m.statevector().reshape(2**tc, 2**tt)
    prob = np.sum(np.abs(v) ** 2, axis=1)
    xs = np.arange(2**tc)
    for y in range(2**tc):
        amp = np.sum(np.exp(2j * np.pi * xs * (phi - y / 2**tc))) / 2**tc
        assert prob[y] == pytest.approx(abs(amp) ** 2, abs=1e-12)


def test_routing_vs_statevector():
    """3x3 grid circuit with vertical couplers routed by SWAP chains, no truncation."""
    ops = circuits.grid_rcs(3, 3, 4, seed=3)
    m = omps.OracleMPS(9, 32)
    m.run(ops)
    v = sv.run(ops, 9)
    assert np.abs(m.statevector() - v).max() < 1e-12


def test_routing_far_pair_both_orders():
    rng = np.random.default_rng(8)
    g = gates.haar_unitary(rng, 4)
    base = circuits.brickwall(6, 2, seed=4)
    for q1, q2 in [(0, 5), (5, 1), (2, 4)]:
        ops = base + [("2q", q1, q2, g)]
        m = omps.OracleMPS(6, 16)
        m.run(ops)
        assert np.abs(m.statevector() - sv.run(ops, 6)).max() < 1e-12


def test_truncation_identity_canon():
    """Under the canonical policy every split removes exactly its discarded weight
    from the norm fidelity: F_after = F_before - delta (Sec. III-E)."""
    n = 10
    ops = circuits.brickwall(n, 10, seed=6)
    m = omps.OracleMPS(n, 6, "canon")
    f = 1.0
    for op in ops:
        if op[0] == "1q":
            m.apply_1q(op[1], op[2])
            continue
        d = m.apply_2q(op[1], op[3])
        f_new = m.norm2()
        assert f_new == pytest.approx(f - d, rel=1e-11, abs=1e-14)
        assert m.centre_norm2() == pytest.approx(f_new, rel=1e-11)
        f = f_new
    assert f < 1.0 and sum(m.discarded) > 0
    assert f == pytest.approx(1.0 - sum(m.discarded), rel=1e-10)


def test_canonical_form_after_moves():
    n = 8
    m = omps.OracleMPS(n, 16, "canon")
    m.run(circuits.brickwall(n, 6, seed=2))
    m.move_centre(3)
    for i, s in enumerate(m.sites):
        cl, _, cr = s.shape
        if i < 3:
            a = s.reshape(2 * cl, cr)
            assert np.abs(a.conj().T @ a - np.eye(cr)).max() < 1e-12
        elif i > 3:
            a = s.reshape(cl, 2 * cr)
            assert np.abs(a @ a.conj().T - np.eye(cl)).max() < 1e-12


def test_norm_fidelity_tracks_overlap_fidelity():
    """Sec. III-E (norm-vs-overlap figure): the norm fidelity approximates the overlap fidelity with
    the exact state, and pivoted QR tends to underestimate it.  The overlap is
    taken with the truncated state normalised, |<E|T>|^2 / <T|T>."""
    n = 12
    ops = circuits.brickwall(n, 12, seed=10)
    exact = sv.run(ops, n)
    for chi in (16, 24, 32):
        m = omps.OracleMPS(n, chi, "canon")
        m.run(ops)
        fbar = m.norm2()
        t = m.statevector()
        fov = abs(np.vdot(exact, t)) ** 2 / fbar
        assert 0 < fbar < 1 and 0 < fov < 1
        assert abs(fbar - fov) < 0.05 * fov
        assert fbar <= fov


def test_random_canonical_state_has_unit_norm():
    n = 10
    bonds = states.max_bond_dims(n, 8)
    sites = states.random_canonical_mps(n, bonds, 4, seed=1)
    m = omps.OracleMPS(n, 8)
    m.set_sites(sites, centre=4)
    assert m.norm2() == pytest.approx(1.0, abs=1e-12)
    assert m.centre_norm2() == pytest.approx(1.0, abs=1e-12)


def test_permute_is_qubit_transposition_without_truncation():
    """Site permutation (bubble sort of SWAPs) without truncation: the state equals the
    statevector with its qubit axes transposed accordingly, and the SWAP count is the
    number of inversions of the permutation (brute force)."""
    n = 6
    rng = np.random.default_rng(41)
    ops = circuits.brickwall(n, 4, seed=5)
    m = omps.OracleMPS(n, 64, "canon")
    m.run(ops)
    v = m.statevector().reshape([2] * n)
    order = list(rng.permutation(n))
    swaps = m.permute(order)
    inversions = sum(1 for a in range(n) for b in range(a + 1, n) if order[a] > order[b])
    assert swaps == inversions
    # position p now holds the qubit that was at position order[p]
    w = np.transpose(v, order).reshape(-1)
    assert np.abs(m.statevector() - w).max() < 1e-12


def test_permute_identity_and_reversal():
    n = 5
    m = omps.OracleMPS(n, 32, "local")
    m.run(circuits.brickwall(n, 3, seed=2))
    v = m.statevector()
    assert m.permute(list(range(n))) == 0
    assert np.abs(m.statevector() - v).max() < 1e-14
    assert m.permute(list(range(n - 1, -1, -1))) == n * (n - 1) // 2
    w = np.transpose(v.reshape([2] * n), list(range(n - 1, -1, -1))).reshape(-1)
    assert np.abs(m.statevector() - w).max() < 1e-12


def test_permuted_grid_circuit_is_the_routed_circuit():
    """The permutation approach to the vertical couplers (Sec. III-D.2): row-snake for
    the horizontal patterns, column-snake for the vertical ones, a site permutation in
    between and one back at the end.  Without truncation it prepares exactly the state
    of the SWAP-routed circuit with the same gates."""
    rows, cols, cyc = 3, 4, 8
    routed = circuits.grid_rcs(rows, cols, cyc, seed=5)
    permuted = circuits.grid_rcs_permuted(rows, cols, cyc, seed=5)
    n = rows * cols
    v = sv.run(routed, n)
    assert np.abs(sv.run(permuted, n) - v).max() < 1e-12
    perms = [op for op in permuted if op[0] == "perm"]
    assert len(perms) == 2  # AB | CDCD | AB: to the column snake and back
    for op in permuted:
        if op[0] == "2q":
            assert abs(op[1] - op[2]) == 1  # every coupler is a chain neighbour
    m = omps.OracleMPS(n, 64, "canon")
    m.run(permuted)
    assert np.abs(m.statevector() - v).max() < 1e-12


def test_embedding_change_swap_counts():
    """2 x 2 grid by hand: row snake (00, 01, 11, 10) to column snake (00, 10, 11, 01)
    is the permutation order = [0, 3, 2, 1], three inversions; the oracle's bubble sort
    applies exactly the inversion count of each embedding change."""
    row = lambda r, c: circuits.snake_position(r, c, 2)  # noqa: E731
    col = lambda r, c: circuits.column_snake_position(r, c, 2)  # noqa: E731
    assert circuits.embedding_change(2, 2, row, col) == [0, 3, 2, 1]
    assert circuits.inversions([0, 3, 2, 1]) == 3
    rows, cols = 3, 3
    row = lambda r, c: circuits.snake_position(r, c, cols)  # noqa: E731
    col = lambda r, c: circuits.column_snake_position(r, c, rows)  # noqa: E731
    order = circuits.embedding_change(rows, cols, row, col)
    m = omps.OracleMPS(rows * cols, 16, "canon")
    m.run(circuits.brickwall(rows * cols, 3, seed=1))
    assert m.permute(order) == circuits.inversions(order) == 15


def test_paper_gate_set_produces_exact_pivot_ties():
    """The random-circuit gate set of App. A (sqrt X / sqrt Y / sqrt W with fSim
    couplers) makes tied column norms common: on a truncated 3 x 4 grid circuit the
    oracle's own splits meet pivot steps whose two largest residual norms (brute-force
    projections) agree to 1e-12.  This is why the GPU's splits of such circuits are
    checked for greedy validity rather than for the oracle's tie-break."""
    from oracle import qr as oqr

    ops = circuits.grid_rcs(3, 4, 8, seed=11, singles="paper")
    ref = omps.OracleMPS(12, 8, "canon")
    ties = 0
    for op in ops:
        if op[0] == "1q":
            ref.apply_1q(op[1], op[2])
            continue
        q1, q2, g = op[1], op[2], np.asarray(op[3])
        if q1 > q2:
            q1, q2, g = q2, q1, omps.SWAP @ g @ omps.SWAP
        seq = [(b, omps.SWAP) for b in range(q1, q2 - 1)] + [(q2 - 1, g)]
        seq += [(b, omps.SWAP) for b in range(q2 - 2, q1 - 1, -1)]
        for i, gg in seq:
            ref.move_centre(i)
            a, b = ref.sites[i], ref.sites[i + 1]
            cl, cm, cr = a.shape[0], a.shape[2], b.shape[2]
            x = (a.reshape(2 * cl, cm) @ b.reshape(cm, 2 * cr)).reshape(cl, 2, 2, cr)
            theta = np.einsum("abcd,lcdr->labr", gg.reshape(2, 2, 2, 2), x).reshape(2 * cl, 2 * cr)
            _, _, p, _ = oqr.cpqr(theta, kmax=8)
            k = min(theta.shape[0], theta.shape[1], 8)
            for j in range(k):
                if j:
                    q = np.linalg.qr(theta[:, p[:j]])[0]
                    res = np.sum(np.abs(theta - q @ (q.conj().T @ theta)) ** 2, axis=0)
                else:
                    res = np.sum(np.abs(theta) ** 2, axis=0)
                res[p[:j]] = -1.0
                top = np.sort(res)[::-1]
                if len(top) > j + 1 and top[0] > 1e-20 and top[0] - top[1] <= 1e-12 * top[0]:
                    ties += 1
            ref.apply_2q(i, gg)
    assert ties > 0


@pytest.mark.parametrize("policy", ["canon", "local"])
def test_permute_layers_is_qubit_transposition_without_truncation(policy):
    """Odd-even transposition sort of SWAPs without truncation: the statevector's axes
    transposed, SWAP count = inversions (brute force), at most n passes, and (under the
    local policy) the same state as the bubble-sort order."""
    n = 7
    rng = np.random.default_rng(43)
    ops = circuits.brickwall(n, 4, seed=6)
    for trial in range(4):
        m = omps.OracleMPS(n, 128, policy)
        m.run(ops)
        v = m.statevector().reshape([2] * n)
        order = list(rng.permutation(n)) if trial else list(range(n))[::-1]
        swaps, passes = m.permute_layers(order)
        inversions = sum(1 for a in range(n) for b in range(a + 1, n) if order[a] > order[b])
        assert swaps == inversions and passes <= n
        assert np.abs(m.statevector() - np.transpose(v, order).reshape(-1)).max() < 1e-12
        if trial == 0:
            assert passes == n  # the reversal needs n passes


def test_permute_layers_passes_are_disjoint_layers():
    """Each pass swaps pairs of one parity only, so the SWAPs of a pass act on disjoint
    bonds (recorded by wrapping the oracle's swap)."""
    n = 9
    order = list(np.random.default_rng(3).permutation(n))
    m = omps.OracleMPS(n, 4, "local")
    seen = []
    orig = m.swap
    m.swap = lambda q, chi=None: (seen.append(q), orig(q, chi))
    m.permute_layers(order)
    # the recorded SWAPs split into runs of one parity, each strictly increasing by >= 2
    i = 0
    while i < len(seen):
        par = seen[i] % 2
        j = i
        while j < len(seen) and seen[j] % 2 == par and (j == i or seen[j] > seen[j - 1]):
            j += 1
        assert all(b - a >= 2 for a, b in zip(seen[i:j], seen[i + 1:j]))
        i = j
