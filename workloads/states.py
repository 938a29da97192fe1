"""Seeded initial site tensors.

Site layout everywhere: site i is a complex array of shape (chi_l, 2, chi_r),
row-major (Sec. III-A.1 flat row-major layout), bond dims chi_0 = chi_n = 1.

The "saturated" input of Sec. III-D.1 fills site entries with random values;
here they are i.i.d. standard complex Gaussians.  Where a site must be an
isometry (left- or right-canonical side of a mixed-canonical state), a random
isometry is generated directly: Haar (QR of a Ginibre matrix) for small
dimensions, and for large ones the product D1 F D2 F D3 of unitary DFTs F and
random diagonal phases D restricted to the needed columns, which costs
O(d^2 log d) instead of the O(d^3) of a QR.
"""

import numpy as np

_HAAR_MAX = 512


def complex_gaussian(rng, shape, dtype=np.complex128):
    z = rng.standard_normal(shape) + 1j * rng.standard_normal(shape)
    return (z / np.sqrt(2.0)).astype(dtype)


def random_isometry(rng, d, c):
    """d x c matrix with orthonormal columns (c <= d)."""
    assert c <= d
    if d <= _HAAR_MAX:
        z = complex_gaussian(rng, (d, c))
        q, r = np.linalg.qr(z)
        ph = np.diag(r) / np.abs(np.diag(r))
        return q * ph[None, :]
    ph = [np.exp(2j * np.pi * rng.random(d)) for _ in range(3)]
    m = np.zeros((d, c), dtype=np.complex128)
    m[np.arange(c), np.arange(c)] = ph[2][:c]
    m = np.fft.fft(m, axis=0, norm="ortho")
    m *= ph[1][:, None]
    m = np.fft.fft(m, axis=0, norm="ortho")
    m *= ph[0][:, None]
    return m


def max_bond_dims(n, chi_max):
    """Largest bond dims reachable on an n-site chain: min(2^b, 2^(n-b), chi_max)."""
    return [min(2**b, 2 ** (n - b), chi_max) for b in range(n + 1)]


def random_canonical_mps(n, bonds, centre, seed, dtype=np.complex128):
    """Random mixed-canonical MPS with the given bond dims and orthogonality centre.

    Sites left of ``centre`` are left-isometries ((chi_l*2) x chi_r with
    orthonormal columns), sites right of it right-isometries (chi_l x (2*chi_r)
    with orthonormal rows), and the centre site holds i.i.d. complex Gaussians
    scaled to unit Frobenius norm, so the state has norm 1.
    """
    assert len(bonds) == n + 1 and bonds[0] == 1 and bonds[n] == 1
    rng = np.random.default_rng(seed)
    sites = []
    for i in range(n):
        cl, cr = bonds[i], bonds[i + 1]
        if i < centre:
            assert cr <= 2 * cl
            s = random_isometry(rng, 2 * cl, cr).reshape(cl, 2, cr)
        elif i > centre:
            assert cl <= 2 * cr
            s = random_isometry(rng, 2 * cr, cl).T.conj().reshape(cl, 2, cr)
        else:
            s = complex_gaussian(rng, (cl, 2, cr))
            s /= np.linalg.norm(s)
        sites.append(np.ascontiguousarray(s, dtype=dtype))
    return sites


def saturated_two_site(chi_l, chi_m, chi_r, seed, dtype=np.complex128):
    """Two neighbouring saturated sites (A, B) with B right-orthonormal.

    A: (chi_l, 2, chi_m) i.i.d. complex Gaussian scaled to unit norm.
    B: (chi_m, 2, chi_r) with orthonormal rows of its chi_m x (2 chi_r) matrix.
    """
    rng = np.random.default_rng(seed)
    a = complex_gaussian(rng, (chi_l, 2, chi_m))
    a /= np.linalg.norm(a)
    b = random_isometry(rng, 2 * chi_r, chi_m).T.conj().reshape(chi_m, 2, chi_r)
    return np.ascontiguousarray(a, dtype=dtype), np.ascontiguousarray(b, dtype=dtype)
