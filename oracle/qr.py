"""ctypes wrapper of the oracle's plain Householder QR (test infrastructure).

See oracle/src/oracle_qr.cpp for the algorithm (Sec. III-B.2, QR with
pivoting M = Q R P^T, truncated after k = min(m, n, kmax) reflectors).
"""

import ctypes

import numpy as np

from . import build as _build

_lib = None


def _load():
    global _lib
    if _lib is None:
        path = _build.build()
        lib = ctypes.CDLL(path)
        lib.oracle_cpqr.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                    ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p,
                                    ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                                    ctypes.POINTER(ctypes.c_double)]
        lib.oracle_cpqr.restype = ctypes.c_int
        lib.oracle_form_q.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_void_p, ctypes.c_int64,
                                      ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64]
        lib.oracle_form_q.restype = ctypes.c_int
        lib.oracle_cpqr_replay.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                           ctypes.POINTER(ctypes.c_int), ctypes.c_void_p, ctypes.c_int64,
                                           ctypes.c_void_p, ctypes.POINTER(ctypes.c_int),
                                           ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_double),
                                           ctypes.c_void_p, ctypes.c_void_p]
        lib.oracle_cpqr_replay.restype = ctypes.c_int
        lib.oracle_num_threads.restype = ctypes.c_int
        _lib = lib
    return _lib


def num_threads():
    return _load().oracle_num_threads()


def factor(a, kmax=None, pivot=True):
    """Householder QR of ``a`` (m x n complex), truncated after kmax reflectors.

    Returns a dict with
      ``w``    : the factored matrix (m x n, column-major content as a Fortran
                 array): R in the first k rows, reflectors below the diagonal;
      ``tau``  : k reflector scalars;
      ``jpvt`` : column permutation, jpvt[t] = original column at position t;
      ``k``    : number of reflectors;
      ``discarded`` : ||trailing block||_F^2 after k steps.
    """
    lib = _load()
    a = np.asfortranarray(a, dtype=np.complex128).copy(order="F")
    m, n = a.shape
    if kmax is None:
        kmax = min(m, n)
    kk = max(min(m, n, kmax), 0)
    tau = np.zeros(max(kk, 1), dtype=np.complex128)
    jpvt = np.zeros(max(n, 1), dtype=np.int32)
    k_out = ctypes.c_int(0)
    disc = ctypes.c_double(0.0)
    rc = lib.oracle_cpqr(m, n, int(kmax), 1 if pivot else 0, a.ctypes.data, max(m, 1),
                         tau.ctypes.data, jpvt.ctypes.data_as(ctypes.POINTER(ctypes.c_int)),
                         ctypes.byref(k_out), ctypes.byref(disc))
    if rc != 0:
        raise ValueError("oracle_cpqr: bad argument")
    k = k_out.value
    return {"w": a, "tau": tau[:k], "jpvt": jpvt[:n].astype(np.int64), "k": k,
            "discarded": disc.value}


def form_q(f):
    """Q[:, :k] (m x k) from a ``factor`` result."""
    lib = _load()
    w = f["w"]
    m = w.shape[0]
    k = f["k"]
    q = np.zeros((m, k), dtype=np.complex128, order="F")
    if k > 0:
        tau = np.ascontiguousarray(f["tau"], dtype=np.complex128)
        rc = lib.oracle_form_q(m, k, w.ctypes.data, max(m, 1), tau.ctypes.data, q.ctypes.data,
                               max(m, 1))
        if rc != 0:
            raise ValueError("oracle_form_q: bad argument")
    return q


def r_factor(f):
    """R (k x n, columns in pivoted order) from a ``factor`` result."""
    k = f["k"]
    return np.triu(f["w"][:k, :])


def cpqr(a, kmax=None, pivot=True):
    """Truncated CPQR: returns (Q (m x k), R (k x n, pivoted order), jpvt, discarded)."""
    f = factor(a, kmax, pivot)
    return form_q(f), r_factor(f), f["jpvt"], f["discarded"]


def replay(a, order, kmax=None):
    """The pivoted factorisation of ``factor`` with the pivot of step j forced to the
    original column ``order[j]`` (j < k).  Returns ``factor``'s dict plus
    ``chosen2`` / ``max2`` (k entries): the exact squared residual norm of the column
    taken at each step and the largest one among the remaining columns.  A pivot
    sequence is greedy where chosen2 >= max2 (up to a tie tolerance)."""
    lib = _load()
    a = np.asfortranarray(a, dtype=np.complex128).copy(order="F")
    m, n = a.shape
    if kmax is None:
        kmax = min(m, n)
    kk = max(min(m, n, kmax), 0)
    order = np.ascontiguousarray(np.asarray(order, dtype=np.int32)[:kk])
    if order.shape[0] < kk:
        raise ValueError("replay: order needs k entries")
    tau = np.zeros(max(kk, 1), dtype=np.complex128)
    jpvt = np.zeros(max(n, 1), dtype=np.int32)
    chosen2 = np.zeros(max(kk, 1))
    max2 = np.zeros(max(kk, 1))
    k_out = ctypes.c_int(0)
    disc = ctypes.c_double(0.0)
    rc = lib.oracle_cpqr_replay(m, n, int(kmax), order.ctypes.data_as(ctypes.POINTER(ctypes.c_int)),
                                a.ctypes.data, max(m, 1), tau.ctypes.data,
                                jpvt.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), ctypes.byref(k_out),
                                ctypes.byref(disc), chosen2.ctypes.data, max2.ctypes.data)
    if rc != 0:
        raise ValueError("oracle_cpqr_replay: bad argument or pivot order")
    k = k_out.value
    return {"w": a, "tau": tau[:k], "jpvt": jpvt[:n].astype(np.int64), "k": k, "discarded": disc.value,
            "chosen2": chosen2[:k], "max2": max2[:k]}


def cpqr_replay(a, order, kmax=None):
    """``replay`` as (Q (m x k), R (k x n, pivoted order), jpvt, discarded, chosen2, max2)."""
    f = replay(a, order, kmax)
    return form_q(f), r_factor(f), f["jpvt"], f["discarded"], f["chosen2"], f["max2"]
