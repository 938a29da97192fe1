"""Seeded synthetic circuits (gate lists).

A circuit is a list of operations:

* ``("1q", q, u)``       one-qubit gate ``u`` (2x2) on qubit position ``q``;
* ``("2q", q1, q2, g)``  two-qubit gate ``g`` (4x4, see ``gates``) on the
  ordered pair of positions (q1, q2).  The positions need not be adjacent; a
  consumer routes non-adjacent pairs with SWAP chains (Sec. III-C.4).
* ``("perm", order)``    site permutation (Sec. III-C.4): afterwards position p
  holds the qubit that was at position order[p].
* ``("mpo", first, ws)`` matrix product operator on positions first ..
  first+len(ws)-1, ws[j] of shape (a, b, 2, 2) = W[left bond, right bond, out, in].

Positions are MPS site indices: site 0 is the most significant bit of the
statevector index (Sec. II-A.1 tensor-product order).
"""

import numpy as np

from . import gates as G


def brickwall(n, depth, seed):
    """Brick-wall circuit of Haar-random gates on a 1D chain.

    Layer t applies a Haar SU(2) gate to every qubit, then Haar SU(4) gates on
    the bonds (2j, 2j+1) for even t and (2j+1, 2j+2) for odd t.
    """
    rng = np.random.default_rng(seed)
    ops = []
    for t in range(depth):
        for q in range(n):
            ops.append(("1q", q, G.haar_unitary(rng, 2)))
        start = 0 if t % 2 == 0 else 1
        for q in range(start, n - 1, 2):
            ops.append(("2q", q, q + 1, G.haar_unitary(rng, 4)))
    return ops


def brickwall_layers(n, depth, seed):
    """Same gates as ``brickwall`` grouped per layer: a list of (ones, twos).

    ``ones`` is a list of (q, u); ``twos`` a list of (q, g) acting on (q, q+1).
    """
    ops = brickwall(n, depth, seed)
    layers = []
    i = 0
    for t in range(depth):
        ones = [(op[1], op[2]) for op in ops[i:i + n]]
        i += n
        start = 0 if t % 2 == 0 else 1
        cnt = len(range(start, n - 1, 2))
        twos = [(op[1], op[3]) for op in ops[i:i + cnt]]
        i += cnt
        layers.append((ones, twos))
    return layers


def ghz(n):
    """GHZ preparation: H on qubit 0 then a CNOT chain (i -> i+1)."""
    ops = [("1q", 0, G.hadamard())]
    for q in range(n - 1):
        ops.append(("2q", q, q + 1, G.cnot()))
    return ops


def basis_state(n, x):
    """X gates preparing |x> from |0...0> (qubit 0 = most significant bit)."""
    ops = []
    for q in range(n):
        if (x >> (n - 1 - q)) & 1:
            ops.append(("1q", q, G.x_gate()))
    return ops


def _cphase_k(k, sign):
    return G.cphase(sign * 2 * np.pi / 2**k)


def qft_noswap(qubits):
    """QFT on the listed positions (first = most significant), final swaps omitted.

    Hadamards and controlled R_k gates of App. A.  Maps |x> to
    prod_j (|0> + exp(2 pi i x 2^j / 2^t) |1>)/sqrt(2) on position qubits[j].
    """
    t = len(qubits)
    ops = []
    for j in range(t):
        ops.append(("1q", qubits[j], G.hadamard()))
        for k in range(2, t - j + 1):
            ops.append(("2q", qubits[j + k - 1], qubits[j], _cphase_k(k, +1)))
    return ops


def iqft_noswap(qubits):
    """Inverse of ``qft_noswap``: the IQFT with R_k^dagger, swaps omitted (App. A)."""
    t = len(qubits)
    ops = []
    for j in range(t - 1, -1, -1):
        for k in range(t - j, 1, -1):
            ops.append(("2q", qubits[j + k - 1], qubits[j], _cphase_k(k, -1)))
        ops.append(("1q", qubits[j], G.hadamard()))
    return ops


def controlled_phase_mpo(phases):
    """MPO (bond 2) of the controlled phases of one control qubit (Sec. III-D.1): the
    control on the first site, targets on the following ones with phase shifts
    diag(1, exp(i phases[k])).  W_first = (Pi_0, Pi_1), W_mid = diag(I, P), W_last =
    (I, P)^T, so the operator is Pi_0 (x) I ... + Pi_1 (x) P_1 (x) P_2 ..."""
    eye = np.eye(2, dtype=np.complex128)
    pi0 = np.diag([1.0, 0.0]).astype(np.complex128)
    pi1 = np.diag([0.0, 1.0]).astype(np.complex128)
    first = np.zeros((1, 2, 2, 2), dtype=np.complex128)
    first[0, 0], first[0, 1] = pi0, pi1
    ws = [first]
    for k, ph in enumerate(phases):
        p = np.diag([1.0, np.exp(1j * ph)]).astype(np.complex128)
        if k < len(phases) - 1:
            w = np.zeros((2, 2, 2, 2), dtype=np.complex128)
            w[0, 0], w[1, 1] = eye, p
        else:
            w = np.zeros((2, 1, 2, 2), dtype=np.complex128)
            w[0, 0], w[1, 0] = eye, p
        ws.append(w)
    return ws


def iqft_mpo(qubits):
    """``iqft_noswap`` with the controlled phases of each qubit merged into one MPO of
    bond 2 (Sec. III-D.1): for j = t-1 .. 0 the MPO on positions qubits[j] ..
    qubits[t-1] (consecutive) with phases -2 pi / 2^k on qubits[j+k-1], then H on
    qubits[j]."""
    t = len(qubits)
    assert list(qubits) == list(range(qubits[0], qubits[0] + t)), "positions must be consecutive"
    ops = []
    for j in range(t - 1, -1, -1):
        if j < t - 1:
            ops.append(("mpo", qubits[j], controlled_phase_mpo([-2 * np.pi / 2**k for k in range(2, t - j + 1)])))
        ops.append(("1q", qubits[j], G.hadamard()))
    return ops


def qpe(n_count, n_target, seed):
    """Quantum phase estimation of a seeded random diagonal unitary.

    U = tensor_i diag(1, exp(i theta_i)) on the target register (positions
    n_count .. n_count+n_target-1), target initialised to a seeded basis state
    |t>, an eigenstate with phase phi = sum_i t_i theta_i / (2 pi) mod 1.
    Counting qubit j controls U^(2^j), decomposed into controlled-phase gates,
    followed by ``iqft_noswap`` on the counting register.  For dyadic phi the
    counting register ends in |phi * 2^n_count> (qubit 0 most significant).

    Returns (ops, phi).
    """
    rng = np.random.default_rng(seed)
    theta = rng.uniform(0, 2 * np.pi, n_target)
    tbits = rng.integers(0, 2, n_target)
    if not tbits.any():
        tbits[0] = 1
    ops = []
    for i in range(n_target):
        if tbits[i]:
            ops.append(("1q", n_count + i, G.x_gate()))
    for j in range(n_count):
        ops.append(("1q", j, G.hadamard()))
    for j in range(n_count):
        for i in range(n_target):
            ang = (2**j * theta[i]) % (2 * np.pi)
            ops.append(("2q", j, n_count + i, G.cphase(ang)))
    ops += iqft_noswap(list(range(n_count)))
    phi = (float(np.dot(tbits, theta)) / (2 * np.pi)) % 1.0
    return ops, phi


def qpe_dyadic(n_count, n_target, seed):
    """QPE as in ``qpe`` with angles chosen so that phi is an n_count-bit fraction."""
    rng = np.random.default_rng(seed)
    tbits = rng.integers(0, 2, n_target)
    tbits[0] = 1
    y = int(rng.integers(0, 2**n_count))
    theta = np.zeros(n_target)
    theta[0] = 2 * np.pi * y / 2**n_count
    ops = []
    for i in range(n_target):
        if tbits[i]:
            ops.append(("1q", n_count + i, G.x_gate()))
    for j in range(n_count):
        ops.append(("1q", j, G.hadamard()))
    for j in range(n_count):
        for i in range(n_target):
            ang = (2**j * theta[i]) % (2 * np.pi)
            ops.append(("2q", j, n_count + i, G.cphase(ang)))
    ops += iqft_noswap(list(range(n_count)))
    return ops, y


def snake_position(r, c, cols):
    """1D MPS position of grid qubit (r, c) in the row-snake embedding."""
    return r * cols + (c if r % 2 == 0 else cols - 1 - c)


def grid_pattern(rows, cols, pat):
    """Coupler list of one interaction pattern on a rows x cols grid.

    A/B: horizontal couplers (r,c)-(r,c+1) with c even / odd.
    C/D: vertical couplers (r,c)-(r+1,c) with r even / odd.
    The paper's Sycamore patterns exist only as figures; this is the grid analogue.
    """
    pairs = []
    if pat in "AB":
        par = 0 if pat == "A" else 1
        for r in range(rows):
            for c in range(par, cols - 1, 2):
                pairs.append(((r, c), (r, c + 1)))
    else:
        par = 0 if pat == "C" else 1
        for r in range(par, rows - 1, 2):
            for c in range(cols):
                pairs.append(((r, c), (r + 1, c)))
    return pairs


def grid_rcs(rows, cols, cycles, seed, pattern="ABCDCDAB", singles="paper"):
    """Random circuit on a rows x cols grid, snaked onto a 1D chain.

    Each cycle: a one-qubit gate drawn i.i.d. uniformly from {sqrt(X), sqrt(Y),
    sqrt(W)} on every qubit (App. A), then fSim on every coupler of the cycle's
    pattern (Eq. (fsim)); patterns follow ``pattern`` cyclically (Sec. III-D.2).
    Vertical couplers are non-adjacent in the snake and need routing.
    ``singles="haar"`` draws Haar SU(2) one-qubit gates instead: the paper's
    gate set makes exactly equal column norms (pivot ties) common, which a
    test comparing two implementations pivot for pivot has to avoid.
    """
    rng = np.random.default_rng(seed)
    paper = [G.sqrt_x(), G.sqrt_y(), G.sqrt_w()]
    f = G.fsim()
    ops = []
    for cyc in range(cycles):
        for r in range(rows):
            for c in range(cols):
                u = paper[int(rng.integers(0, 3))] if singles == "paper" else G.haar_unitary(rng, 2)
                ops.append(("1q", snake_position(r, c, cols), u))
        pat = pattern[cyc % len(pattern)]
        for (a, b) in grid_pattern(rows, cols, pat):
            pa = snake_position(a[0], a[1], cols)
            pb = snake_position(b[0], b[1], cols)
            ops.append(("2q", pa, pb, f))
    return ops


def column_snake_position(r, c, rows):
    """1D position of grid qubit (r, c) in the column-snake embedding, where the
    vertical couplers (r, c)-(r+1, c) are chain neighbours."""
    return c * rows + (r if c % 2 == 0 else rows - 1 - r)


def embedding_change(rows, cols, cur, new):
    """order of the site permutation from embedding ``cur`` to ``new`` (each a
    function (r, c) -> position): new position p receives the qubit now at order[p]."""
    order = [0] * (rows * cols)
    for r in range(rows):
        for c in range(cols):
            order[new(r, c)] = cur(r, c)
    return order


def grid_rcs_permuted(rows, cols, cycles, seed, pattern="ABCDCDAB", singles="paper"):
    """The circuit of ``grid_rcs`` (same seed, same gates) with the paper's
    permutation approach to the vertical couplers (Sec. III-D.2): horizontal
    patterns (A, B) run in the row-snake embedding and vertical ones (C, D) in the
    column-snake embedding, where every coupler is a nearest-neighbour pair; a
    ("perm", order) layer changes the embedding between them, and a last one
    restores the row snake, so the final state is that of ``grid_rcs``."""
    rng = np.random.default_rng(seed)
    paper = [G.sqrt_x(), G.sqrt_y(), G.sqrt_w()]
    f = G.fsim()
    row = lambda r, c: snake_position(r, c, cols)  # noqa: E731
    col = lambda r, c: column_snake_position(r, c, rows)  # noqa: E731
    cur = row
    ops = []
    for cyc in range(cycles):
        pat = pattern[cyc % len(pattern)]
        want = row if pat in "AB" else col
        for r in range(rows):
            for c in range(cols):
                u = paper[int(rng.integers(0, 3))] if singles == "paper" else G.haar_unitary(rng, 2)
                ops.append(("1q", cur(r, c), u))
        if want is not cur:
            ops.append(("perm", embedding_change(rows, cols, cur, want)))
            cur = want
        for (a, b) in grid_pattern(rows, cols, pat):
            ops.append(("2q", cur(*a), cur(*b), f))
    if cur is not row:
        ops.append(("perm", embedding_change(rows, cols, cur, row)))
    return ops


def inversions(order):
    """Number of pairs p < q with order[p] > order[q]: the SWAP count of a bubble sort."""
    return sum(1 for p in range(len(order)) for q in range(p + 1, len(order)) if order[p] > order[q])


def count_two_qubit(ops):
    return sum(1 for op in ops if op[0] == "2q")
