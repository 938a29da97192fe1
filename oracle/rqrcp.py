"""Truncated QR with randomized column pivoting (test infrastructure).

ORACLE -- slow, plain, complex128.  Only tests, the package smoke check and the
benchmark's CPU legs use it; the GPU library never calls it.

The paper truncates a bond by a column-pivoted QR (Sec. III-B.2, M = Q R P^T) and
cites improvements to the QR in its bond-truncation discussion (Sec. IV-A.1).  This
module restates one such improvement, blocked QR with randomized column pivoting
(RQRCP: P. Duersch and M. Gu, "Randomized QR with column pivoting", SIAM J. Sci.
Comput. 39 (2017); P.-G. Martinsson, G. Quintana-Orti, N. Heavner and R. van de
Geijn, "Householder QR factorization with randomization for column pivoting
(HQRRP)", SIAM J. Sci. Comput. 39 (2017)).  Pivots are chosen on a small sketch
Y = Omega A instead of on A itself, so the factorisation of A needs no per-pivot
pass over the trailing matrix.  For a matrix A (m x n), a block size nb, an
oversampling p and k = min(m, n, kmax):

  1. Y = Omega A with Omega an (nb + p) x m sketching matrix (here: entries
     +-1 from a counter-based generator, ``sketch_signs``).
  2. For each block j0 = 0, nb, 2 nb, ... < k, of width kb = min(nb, k - j0):
     a. kb steps of the plain column-pivoted QR (oracle/qr.py) of the sketch's
        remaining columns Y[:, j0:] choose the block's pivots; the resulting
        column permutation is applied to A[:, j0:], Y[:, j0:] and jpvt;
     b. kb unpivoted Householder steps on A[j0:, j0:] (the same reflector
        convention as oracle/qr.py), which leave R11 = A[j0:J1, j0:J1] and
        R12 = A[j0:J1, J1:] (J1 = j0 + kb) and the updated trailing block;
     c. sketch update Y[:, J1:] -= (Y[:, j0:J1] R11^{-1}) R12 (Duersch and Gu):
        the updated sketch is Omega Q2 times the trailing block A[J1:, J1:], where
        Q2 spans the columns of Q after the first J1.  A diagonal entry of R11 that
        is zero (or below the smallest normal number: a column with no residual)
        contributes nothing: its column of Y R11^{-1} is set to zero.
  3. R = the first k rows, Q[:, :k] = H_0 ... H_{k-1} I, and the discarded weight
     is ||A[k:, k:]||_F^2.

With Omega an m x m unitary the sketch has the residual norms of A itself, so the
pivots are those of the plain column-pivoted QR (a pin of the sketch update).
"""

import numpy as np

from . import qr as _qr

_M64 = (1 << 64) - 1
_GOLDEN = 0x9E3779B97F4A7C15


def splitmix64(counters, seed):
    """SplitMix64 (G. L. Steele, D. Lea and C. H. Flood, "Fast splittable pseudorandom
    number generators", OOPSLA 2014) as a counter-based generator: output number c of
    the generator started at state `seed`, i.e. the mixing function applied to
    seed + (c + 1) * 0x9E3779B97F4A7C15 (mod 2^64).  uint64 in, uint64 out."""
    c = np.asarray(counters, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(seed & _M64) + (c + np.uint64(1)) * np.uint64(_GOLDEN)
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        z = z ^ (z >> np.uint64(31))
    return z


def sketch_signs(rows, m, seed):
    """The rows x m sketching matrix: entry (i, r) is -1 when the top bit of SplitMix64
    output number i*m + r (generator state `seed`) is set, else +1."""
    c = np.arange(rows * m, dtype=np.uint64)
    bits = splitmix64(c, seed) >> np.uint64(63)
    return np.where(bits.reshape(rows, m) == 1, -1.0, 1.0).astype(np.complex128)


def rqrcp(a, kmax=None, seed=0, nb=64, oversample=8, omega=None, keep_sketches=False):
    """Truncated RQRCP of ``a`` (m x n), blocks of ``nb`` pivots and an ``nb + oversample``
    row sketch (defaults: 64 and 8, the GPU library's blocks of two 32-column panels).  Returns a dict with ``q`` (m x k), ``r`` (k x n,
    columns in pivoted order), ``jpvt`` (jpvt[t] = original column at position t),
    ``discarded`` (||A[k:, k:]||_F^2), and with ``keep_sketches`` the sketch and the
    column order after every block.  ``omega`` replaces the sketching matrix (any l x m)."""
    a = np.array(a, dtype=np.complex128)
    m, n = a.shape
    k = min(m, n, n if kmax is None else kmax)
    om = sketch_signs(nb + oversample, m, seed) if omega is None else np.asarray(omega, dtype=np.complex128)
    y = om @ a
    jpvt = np.arange(n)
    tau = np.zeros(max(k, 1), dtype=np.complex128)
    sketches = []
    tiny = np.finfo(np.float64).tiny
    for j0 in range(0, k, nb):
        kb = min(nb, k - j0)
        j1 = j0 + kb
        # a. pivots of this block from the sketch
        f = _qr.factor(y[:, j0:], kmax=kb, pivot=True)
        perm = f["jpvt"]
        a[:, j0:] = a[:, j0:][:, perm]
        y[:, j0:] = y[:, j0:][:, perm]
        jpvt[j0:] = jpvt[j0:][perm]
        # b. kb unpivoted Householder steps on the trailing matrix
        g = _qr.factor(a[j0:, j0:], kmax=kb, pivot=False)
        a[j0:, j0:] = g["w"]
        tau[j0:j1] = g["tau"]
        # c. sketch update with the pseudo-inverse rule for zero diagonal entries
        r11 = np.triu(a[j0:j1, j0:j1])
        r12 = a[j0:j1, j1:]
        s = np.zeros((y.shape[0], kb), dtype=np.complex128)
        for c in range(kb):  # s R11 = Y[:, j0:j1], column by column (forward substitution)
            rhs = y[:, j0 + c] - s[:, :c] @ r11[:c, c]
            d = r11[c, c]
            s[:, c] = 0.0 if abs(d) ** 2 < tiny else rhs / d
        y[:, j1:] -= s @ r12
        if keep_sketches:
            sketches.append((y.copy(), jpvt.copy()))
    fq = {"w": np.asfortranarray(a), "tau": tau[:k], "k": k}
    q = _qr.form_q(fq)
    r = np.triu(a[:k, :])
    disc = float(np.sum(np.abs(a[k:, k:]) ** 2))
    out = {"q": q, "r": r, "jpvt": jpvt, "discarded": disc, "k": k}
    if keep_sketches:
        out["sketches"] = sketches
    return out
