"""Tensor-core (tcgen05, 3xTF32) complex64 GEMM.

The 3xTF32 split is good to about 3e-7 of the largest entry per K-step of 8.  The
tensor cores' own FP32 accumulation does not round to nearest; accumulated over
the whole K range its error grew linearly with K (measured on GB300: 6e-5 of the
largest entry at K = 4096).  The kernel therefore adds every K-step's TMEM partial
sum into FP32 registers with round-to-nearest adds, like the CUDA-core GEMM, so the
difference between the two grows at most like a random walk: the bar is
|diff| <= 2e-6 * max|ref| * max(1, sqrt(K / 64)) (1.6e-5 at K = 4096, which the
whole-K accumulation failed by 4x).  The split that uses these products is checked
against the FP64 oracle as well.
"""

import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__

    __graft_entry__.build()
    from paper_2505_06119_gb300 import _lib

    return _lib.load()


def run(lib, M, N, K, a_row=1, a_conj=0, a_mask=0, b_row=1, b_conj=0, b_mask=0, theta=0, seed=1):
    e = ctypes.c_double()
    r = ctypes.c_double()
    rc = lib.mps_selftest_gemm(M, N, K, a_row, a_conj, a_mask, b_row, b_conj, b_mask, theta, seed,
                               ctypes.byref(e), ctypes.byref(r))
    assert rc == 0
    return e.value, r.value


def bar(K, ref):
    return 2e-6 * ref * max(1.0, np.sqrt(K / 64))


@pytest.mark.parametrize("M,N,K", [(128, 64, 32), (256, 128, 64), (200, 90, 37), (64, 32, 8), (1000, 333, 517)])
@pytest.mark.parametrize("a_row,b_row", [(1, 1), (0, 0), (1, 0), (0, 1)])
def test_layouts(lib, M, N, K, a_row, b_row):
    err, ref = run(lib, M, N, K, a_row=a_row, b_row=b_row, seed=M + N + K)
    assert err <= bar(K, ref), (err, ref)


@pytest.mark.parametrize("a_conj,b_conj,a_mask,b_mask", [(1, 0, 0, 0), (0, 1, 0, 0), (1, 1, 1, 0), (0, 0, 2, 1),
                                                          (1, 0, 2, 2)])
def test_conj_and_masks(lib, a_conj, b_conj, a_mask, b_mask):
    err, ref = run(lib, 300, 200, 160, a_row=0, b_row=1, a_conj=a_conj, b_conj=b_conj, a_mask=a_mask,
                   b_mask=b_mask, seed=7)
    assert err <= bar(160, ref), (err, ref)


@pytest.mark.parametrize("cl,cr,cm", [(64, 32, 64), (65, 40, 33), (256, 256, 256), (100, 7, 512)])
def test_theta_epilogue(lib, cl, cr, cm):
    err, ref = run(lib, cl, cr, cm, theta=1, seed=cl * cr)
    assert err <= bar(cm, ref), (err, ref)


@pytest.mark.parametrize("K", [1024, 4096])
def test_long_contractions_stay_at_fp32_accuracy(lib, K):
    """Long K (the theta contraction at chi = 1024 and 4096): the error no longer grows
    linearly with K."""
    err, ref = run(lib, 256, 128, K, a_row=1, b_row=1, seed=K)
    assert err <= bar(K, ref), (err, ref)
    err, ref = run(lib, 128, 64, K, theta=1, seed=K + 1)
    assert err <= bar(K, ref), (err, ref)


@pytest.mark.parametrize("cl,cm,cr,chi", [(130, 70, 129, 128), (256, 512, 256, 256)])
def test_mixed_split_with_tensor_cores_matches_oracle(cl, cm, cr, chi):
    """A mixed-precision split whose theta contraction runs on the tensor cores, against
    the FP64 oracle: the kept state Q R P^T to 2e-5 relative, Q orthonormal to 1e-5 (the
    bars of the CUDA-core mixed split)."""
    from oracle import qr as oqr
    from paper_2505_06119_gb300 import MPS
    from workloads import gates, states

    rng = np.random.default_rng(cl + cr + cm)
    a = states.complex_gaussian(rng, (cl, 2, cm)) / np.sqrt(cm)
    b = states.complex_gaussian(rng, (cm, 2, cr))
    g = gates.haar_unitary(rng, 4)
    with MPS(22, 512, precision="mixed", policy="local", tensor_cores=True) as m:
        m.set_site(10, a.astype(np.complex64))
        m.set_site(11, b.astype(np.complex64))
        m.apply_2q(10, g, chi)
        qa, rb = m.get_site(10), m.get_site(11)
    x = (a.reshape(2 * cl, cm) @ b.reshape(cm, 2 * cr)).reshape(cl, 2, 2, cr)
    theta = np.einsum("abcd,lcdr->labr", g.reshape(2, 2, 2, 2), x).reshape(2 * cl, 2 * cr)
    q, r, p, _ = oqr.cpqr(theta, kmax=chi)
    right = np.zeros((chi, 2 * cr), dtype=np.complex128)
    right[:, p] = r
    kept = qa.reshape(2 * cl, -1) @ rb.reshape(rb.shape[0], -1)
    ref = q @ right
    assert np.linalg.norm(kept - ref) / np.linalg.norm(ref) < 2e-5
    qq = qa.reshape(2 * cl, -1)
    assert np.abs(qq.conj().T @ qq - np.eye(qq.shape[1])).max() < 1e-5
