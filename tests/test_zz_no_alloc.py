"""The allocation-free two-site call against the ordinary one.

mps_two_site_apply_noalloc serves callers that may not allocate device
memory (code running inside another component's memory manager, or under a
fixed memory budget): it runs the same two-site gate application as
mps_two_site_apply but takes its scratch space from a fixed array inside the
library.  Its results must equal those of mps_two_site_apply with a
caller-provided workspace, on consecutive calls that reuse the array.  This
file is collected last on purpose.
"""

import ctypes

import numpy as np
import pytest

from workloads import gates, states

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch

    import __graft_entry__

    __graft_entry__.build()
    from paper_2505_06119_gb300 import _lib

    return torch, _lib, _lib.load()


def _apply(env, prec, a, b, g, chi, noalloc):
    torch, L, lib = env
    from paper_2505_06119_gb300.mps import _gate

    code = L.MPS_PREC_FP64 if prec == "fp64" else L.MPS_PREC_MIXED
    dt = torch.complex128 if prec == "fp64" else torch.complex64
    dev = torch.device("cuda:0")
    cl, cm, cr = a.shape[0], a.shape[2], b.shape[2]
    k = min(2 * cl, 2 * cr, chi)
    ta = torch.from_numpy(a).to(dev, dt)
    tb = torch.from_numpy(b).to(dev, dt)
    oa = torch.full((cl, 2, k), 7.0, dtype=dt, device=dev)  # garbage that must be overwritten
    ob = torch.full((k, 2, cr), 7.0, dtype=dt, device=dev)
    disc = torch.full((1,), -1.0, dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream().cuda_stream
    if noalloc:
        rc = lib.mps_two_site_apply_noalloc(code, cl, cm, cr, chi, ta.data_ptr(), tb.data_ptr(), _gate(g, 16),
                                            oa.data_ptr(), ob.data_ptr(), disc.data_ptr(), stream)
    else:
        sz = ctypes.c_size_t()
        assert lib.mps_two_site_workspace(code, cl, cm, cr, chi, ctypes.byref(sz)) == 0
        ws = torch.empty(sz.value + 256, dtype=torch.uint8, device=dev)
        base = (ws.data_ptr() + 255) // 256 * 256
        rc = lib.mps_two_site_apply(code, cl, cm, cr, chi, ta.data_ptr(), tb.data_ptr(), _gate(g, 16),
                                    oa.data_ptr(), ob.data_ptr(), disc.data_ptr(), base, sz.value, stream)
    assert rc == 0
    torch.cuda.synchronize()
    return oa.cpu().numpy(), ob.cpu().numpy(), disc.item()


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-12), ("mixed", 1e-5)])
def test_noalloc_matches_workspace_call_twice(env, prec, tol):
    rng = np.random.default_rng(11)
    cases = [(33, 20, 17, 24), (64, 64, 64, 48)]  # two calls in a row, different shapes and data
    for cl, cm, cr, chi in cases:
        a = states.complex_gaussian(rng, (cl, 2, cm))
        b = states.complex_gaussian(rng, (cm, 2, cr))
        g = gates.haar_unitary(rng, 4)
        ra, rb, rd = _apply(env, prec, a, b, g, chi, noalloc=False)
        na, nb_, nd = _apply(env, prec, a, b, g, chi, noalloc=True)
        assert np.abs(na - ra).max() <= tol
        assert np.abs(nb_ - rb).max() <= tol * max(1.0, np.abs(rb).max())
        assert nd == pytest.approx(rd, rel=1e-9 if prec == "fp64" else 1e-5)


def test_noalloc_rejects_oversized_problem(env):
    torch, L, lib = env
    sz = ctypes.c_size_t()
    assert lib.mps_two_site_workspace(L.MPS_PREC_FP64, 1024, 1024, 1024, 1024, ctypes.byref(sz)) == 0
    assert sz.value > L.MPS_NOALLOC_SCRATCH_BYTES
    g = (L.mps_c128 * 16)()
    rc = lib.mps_two_site_apply_noalloc(L.MPS_PREC_FP64, 1024, 1024, 1024, 1024, 1, 1, g, 1, 1, None, None)
    assert rc == L.MPS_E_UNSUPPORTED


def test_noalloc_allocates_no_device_memory(env):
    """After a first call on the device (which looks up the array's address),
    further calls leave the device's free memory and PyTorch's allocation count
    unchanged: every byte of scratch comes from the library's fixed array."""
    torch, L, lib = env
    from paper_2505_06119_gb300.mps import _gate

    rng = np.random.default_rng(12)
    dev = torch.device("cuda:0")
    cl, cm, cr, chi = 40, 32, 36, 48
    k = min(2 * cl, 2 * cr, chi)
    ta = torch.from_numpy(states.complex_gaussian(rng, (cl, 2, cm)).astype(np.complex64)).to(dev)
    tb = torch.from_numpy(states.complex_gaussian(rng, (cm, 2, cr)).astype(np.complex64)).to(dev)
    oa = torch.empty((cl, 2, k), dtype=torch.complex64, device=dev)
    ob = torch.empty((k, 2, cr), dtype=torch.complex64, device=dev)
    disc = torch.zeros(1, dtype=torch.float64, device=dev)
    g = _gate(gates.haar_unitary(rng, 4), 16)
    stream = torch.cuda.current_stream().cuda_stream

    def call():
        rc = lib.mps_two_site_apply_noalloc(L.MPS_PREC_MIXED, cl, cm, cr, chi, ta.data_ptr(), tb.data_ptr(), g,
                                            oa.data_ptr(), ob.data_ptr(), disc.data_ptr(), stream)
        assert rc == 0

    call()
    torch.cuda.synchronize()
    free0, alloc0 = torch.cuda.mem_get_info(0)[0], torch.cuda.memory_allocated(0)
    for _ in range(5):
        call()
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info(0)[0] == free0
    assert torch.cuda.memory_allocated(0) == alloc0
    assert np.isfinite(disc.item())
