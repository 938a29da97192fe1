"""Tensor-core (tcgen05, 3xTF32) complex64 GEMM against the CUDA-core FP32 GEMM.

The 3xTF32 split is good to about 3e-7 of the largest entry per K-step of 8,
and the tensor cores' FP32 accumulation adds an error that grows linearly
with K (measured on GB300: 7e-7 at K = 32, 1.6e-5 at K = 1024, 6e-5 at
K = 4096, relative to the largest entry).  The bar follows that growth:
|diff| <= 2e-6 * max|ref| * max(1, K / 64).
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
    return 2e-6 * ref * max(1.0, K / 64)


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
