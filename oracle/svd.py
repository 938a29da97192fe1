"""Truncated singular value decomposition split of a two-site block (test infrastructure).

ORACLE: only the tests, the package smoke check and the benchmark's CPU-baseline
leg use it.  The paper lists the SVD M = U S V^dagger next to pivoted QR as a
truncating decomposition (Sec. III-B.2, Table III) and compares the two for bond
truncation (Sec. IV-A.1); the SVD of the reshaped two-site state is its Schmidt
decomposition (Sec. II-A.2).  With theta = U S V^dagger (singular values in
non-increasing order) the split keeps the k = min(m, n, chi_max) largest:

    left  = U[:, :k]                     (an isometry, the left site)
    right = diag(S[:k]) V^dagger[:k, :]  (carries the norm, the right site)
    discarded = sum_{j >= k} S[j]^2

which is the best rank-k approximation of theta in the Frobenius norm (Eckart-Young),
so the discarded weight is the smallest any rank-k split can reach.  The SVD itself
is LAPACK's, through NumPy.
"""

import numpy as np


def svd_split(theta, kmax):
    """Returns (left m x k, right k x n, singular values (all), discarded weight)."""
    theta = np.asarray(theta, dtype=np.complex128)
    m, n = theta.shape
    k = min(m, n, int(kmax))
    u, s, vh = np.linalg.svd(theta, full_matrices=False)
    left = np.ascontiguousarray(u[:, :k])
    right = np.ascontiguousarray(s[:k, None] * vh[:k, :])
    disc = float(np.sum(s[k:] ** 2))
    return left, right, s, disc
