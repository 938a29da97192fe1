"""Gate matrices used by the synthetic circuits.

Conventions (shared by every consumer of this module):

* A one-qubit gate ``u`` is a 2x2 complex128 array, ``u[out, in]``.
* A two-qubit gate ``g`` on the ordered pair (q1, q2) is a 4x4 complex128
  array with row index ``2*a + b`` (outputs) and column index ``2*c + d``
  (inputs), where ``a``/``c`` label qubit q1 and ``b``/``d`` label qubit q2.
  This matches the tensor-product ordering of Sec. II-A.1 (the left factor is
  the more significant bit).

The fixed gates are the ones printed in the paper: the Hadamard and phase gate
R_k of the IQFT appendix (App. A), the three square-root gates of the RCS
appendix (App. A) and the fSim gate of Eq. (fsim) in Sec. III-D.2.
"""

import numpy as np

SQ2 = np.sqrt(2.0)


def hadamard():
    """Hadamard gate, App. A (IQFT gates)."""
    return np.array([[1, 1], [1, -1]], dtype=np.complex128) / SQ2


def r_k(k):
    """Phase gate R_k = diag(1, exp(2 pi i / 2^k)), App. A."""
    return np.array([[1, 0], [0, np.exp(2j * np.pi / 2**k)]], dtype=np.complex128)


def sqrt_x():
    """X^{1/2} as printed in App. A (RCS gates)."""
    return np.array([[1, -1j], [-1j, 1]], dtype=np.complex128) / SQ2


def sqrt_y():
    """Y^{1/2} as printed in App. A (RCS gates)."""
    return np.array([[1, -1], [1, 1]], dtype=np.complex128) / SQ2


def sqrt_w():
    """W^{1/2} as printed in App. A (RCS gates)."""
    w = 1.0 / SQ2
    return np.array([[1, -(1 + 1j) * w], [(1 - 1j) * w, 1]], dtype=np.complex128) / SQ2


def fsim():
    """fSim(theta=pi/2, phi=pi/6) as printed in Eq. (fsim), Sec. III-D.2.

    The MPO form in the same section carries exp(+i pi/6) on the |11> element;
    the equation's exp(-i pi/6) is the one used here.
    """
    g = np.zeros((4, 4), dtype=np.complex128)
    g[0, 0] = 1
    g[1, 2] = -1j
    g[2, 1] = -1j
    g[3, 3] = np.exp(-1j * np.pi / 6)
    return g


def swap():
    """SWAP of the two qubits: |ab> -> |ba> (site permutation, Sec. III-C.4)."""
    g = np.zeros((4, 4), dtype=np.complex128)
    for a in range(2):
        for b in range(2):
            g[2 * b + a, 2 * a + b] = 1
    return g


def cnot():
    """CNOT with control q1 and target q2."""
    g = np.eye(4, dtype=np.complex128)
    g[2:, 2:] = [[0, 1], [1, 0]]
    return g


def cphase(phi):
    """Controlled phase diag(1, 1, 1, exp(i phi)) (symmetric in the two qubits)."""
    return np.diag([1, 1, 1, np.exp(1j * phi)]).astype(np.complex128)


def x_gate():
    return np.array([[0, 1], [1, 0]], dtype=np.complex128)


def haar_unitary(rng, d):
    """Haar-random element of SU(d).

    QR of a complex Ginibre matrix with the phases of R's diagonal moved into Q
    (Mezzadri's recipe), then divided by a d-th root of the determinant.
    """
    z = (rng.standard_normal((d, d)) + 1j * rng.standard_normal((d, d))) / SQ2
    q, r = np.linalg.qr(z)
    ph = np.diag(r) / np.abs(np.diag(r))
    q = q * ph[None, :]
    det = np.linalg.det(q)
    return q / det ** (1.0 / d)


def swap_qubits_of(g):
    """The same 4x4 gate expressed with its two qubits listed in the other order."""
    s = swap()
    return s @ g @ s
