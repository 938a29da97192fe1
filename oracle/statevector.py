"""Brute-force statevector evolution (the oracle's own check, n <= ~16).

ORACLE — test infrastructure.  The state is the 2^n vector of Sec. II-A.1 with
qubit 0 as the most significant bit of the index; gates act as in Sec. II-A.2.
No truncation, no MPS: the exact state a circuit produces.
"""

import numpy as np


def zero_state(n):
    v = np.zeros(2**n, dtype=np.complex128)
    v[0] = 1.0
    return v


def apply_1q(v, n, q, u):
    t = v.reshape(2**q, 2, 2 ** (n - q - 1))
    return np.einsum("ab,xby->xay", np.asarray(u), t).reshape(-1)


def apply_2q(v, n, q1, q2, g):
    """Gate g (row 2a+b, col 2c+d) with a on qubit q1 and b on qubit q2."""
    t = v.reshape([2] * n)
    g4 = np.asarray(g).reshape(2, 2, 2, 2)
    t = np.tensordot(g4, t, axes=([2, 3], [q1, q2]))  # axes: a, b, rest...
    rest = [i for i in range(n) if i not in (q1, q2)]
    order = [0] * n
    order[q1] = 0
    order[q2] = 1
    for pos, ax in enumerate(rest):
        order[ax] = pos + 2
    return np.transpose(t, order).reshape(-1)


def permute(v, n, order):
    """Qubit permutation: axis p of the result is axis order[p] of v."""
    return np.transpose(v.reshape([2] * n), list(order)).reshape(-1)


def mpo_matrix(ws):
    """Dense operator of an MPO (W[a, b, out, in] per site, first site most
    significant): sum over the bonds of the tensor products of W[a, b]."""
    m = np.asarray(ws[0])[0]  # (b, out, in)
    for w in ws[1:]:
        w = np.asarray(w)
        m = np.einsum("bxy,bczw->cxzyw", m, w)
        d = m.shape[1] * m.shape[2]
        m = m.reshape(w.shape[1], d, d)
    return m[0]


def apply_mpo(v, n, first, ws):
    """MPO on the qubits first .. first+len(ws)-1 as a dense operator."""
    L = len(ws)
    t = v.reshape(2**first, 2**L, 2 ** (n - first - L))
    return np.einsum("ab,xby->xay", mpo_matrix(ws), t).reshape(-1)


def run(ops, n, v=None):
    if v is None:
        v = zero_state(n)
    for op in ops:
        if op[0] == "1q":
            v = apply_1q(v, n, op[1], op[2])
        elif op[0] == "perm":
            v = permute(v, n, op[1])
        elif op[0] == "mpo":
            v = apply_mpo(v, n, op[1], op[2])
        else:
            v = apply_2q(v, n, op[1], op[2], op[3])
    return v
