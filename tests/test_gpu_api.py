"""GPU checks of the ABI's non-arithmetic behaviour: the raw-pointer two-site
call on caller-owned (PyTorch) buffers, the optional device allocator, the
bounded-wait error path, and launch accounting."""

import ctypes

import numpy as np
import pytest

from workloads import gates, states

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__

    __graft_entry__.build()


def test_raw_two_site_call_matches_handle_path():
    import torch

    from paper_2505_06119_gb300 import MPS, _lib as L
    from paper_2505_06119_gb300.mps import _gate

    lib = L.load()
    rng = np.random.default_rng(3)
    cl, cm, cr, chi = 33, 20, 17, 24
    a = states.complex_gaussian(rng, (cl, 2, cm))
    b = states.complex_gaussian(rng, (cm, 2, cr))
    g = gates.haar_unitary(rng, 4)
    for prec, dt, tdt in (("fp64", np.complex128, torch.complex128), ("mixed", np.complex64, torch.complex64)):
        code = L.MPS_PREC_FP64 if prec == "fp64" else L.MPS_PREC_MIXED
        dev = torch.device("cuda:0")
        ta = torch.from_numpy(a.astype(dt)).to(dev)
        tb = torch.from_numpy(b.astype(dt)).to(dev)
        k = min(2 * cl, 2 * cr, chi)
        oa = torch.empty((cl, 2, k), dtype=tdt, device=dev)
        ob = torch.empty((k, 2, cr), dtype=tdt, device=dev)
        disc = torch.zeros(1, dtype=torch.float64, device=dev)
        sz = ctypes.c_size_t()
        assert lib.mps_two_site_workspace(code, cl, cm, cr, chi, ctypes.byref(sz)) == 0
        ws = torch.empty(sz.value + 256, dtype=torch.uint8, device=dev)
        base = (ws.data_ptr() + 255) // 256 * 256
        stream = torch.cuda.current_stream().cuda_stream
        rc = lib.mps_two_site_apply(code, cl, cm, cr, chi, ta.data_ptr(), tb.data_ptr(), _gate(g, 16),
                                    oa.data_ptr(), ob.data_ptr(), disc.data_ptr(), base, sz.value, stream)
        assert rc == 0
        torch.cuda.synchronize()
        with MPS(16, max(cl, cm, cr, chi), precision=prec, policy="local") as m:
            m.set_site(7, a)  # reserved bonds at 7, 8, 9 are >= 64
            m.set_site(8, b)
            m.apply_2q(7, g, chi)
            ha, hb = m.get_site(7), m.get_site(8)
            hd, _ = m.discarded()
        tol = 1e-12 if prec == "fp64" else 1e-5
        assert np.abs(oa.cpu().numpy() - ha).max() <= tol
        assert np.abs(ob.cpu().numpy() - hb).max() <= tol * max(1, np.abs(hb).max())
        assert disc.item() == pytest.approx(hd, rel=1e-6)


def test_allocator_hook_and_nomem():
    import torch

    from paper_2505_06119_gb300 import _lib as L

    lib = L.load()
    live = {}

    def alloc(size, ctx):
        p = torch.cuda.caching_allocator_alloc(size, 0, torch.cuda.current_stream())
        live[p] = size
        return p

    def free(p, ctx):
        live.pop(p)
        torch.cuda.caching_allocator_delete(p)

    fa, ff = L.ALLOC_FN(alloc), L.FREE_FN(free)
    cfg = L.mps_config()
    lib.mps_config_init(ctypes.byref(cfg))
    cfg.alloc, cfg.free = fa, ff
    h = ctypes.c_void_p()
    assert lib.mps_create_ex(ctypes.byref(h), 8, 8, ctypes.byref(cfg)) == 0
    assert len(live) > 0
    u = (L.mps_c128 * 4)()
    hg = gates.hadamard().reshape(-1)
    for i in range(4):
        u[i].re, u[i].im = hg[i].real, hg[i].imag
    assert lib.mps_apply_1q(h, 0, u) == 0
    assert lib.mps_swap(h, 0, 0) == 0
    assert lib.mps_sync(h) == 0
    assert lib.mps_destroy(h) == 0
    assert live == {}

    calls = {"n": 0}

    def failing(size, ctx):
        calls["n"] += 1
        if calls["n"] >= 2:
            return None
        return alloc(size, ctx)

    fa2 = L.ALLOC_FN(failing)
    cfg.alloc = fa2
    assert lib.mps_create_ex(ctypes.byref(h), 8, 8, ctypes.byref(cfg)) == L.MPS_E_NOMEM
    assert live == {}


def test_bounded_wait_expiry_is_reported_and_context_survives():
    """A grid barrier told to wait for one CTA too many gives up after the
    configured limit; the call reports MPS_E_TIMEOUT, the handle refuses further
    work, and a fresh handle on the same context works."""
    from paper_2505_06119_gb300 import MPS, MPSError, _lib as L

    m = MPS(6, 8, precision="fp64", wait_timeout_s=0.05, debug_barrier_extra=1)
    m.apply_2q(0, gates.haar_unitary(np.random.default_rng(0), 4))
    with pytest.raises(MPSError) as ei:
        m.sync()
    assert ei.value.code == L.MPS_E_TIMEOUT
    with pytest.raises(MPSError) as ei:
        m.apply_1q(0, gates.hadamard())
    assert ei.value.code == L.MPS_E_STATE
    m.close()
    with MPS(6, 8, precision="fp64") as m2:
        m2.apply_1q(0, gates.hadamard())
        m2.apply_2q(0, gates.cnot())
        assert abs(m2.amplitude([1, 1, 0, 0, 0, 0]) - 1 / np.sqrt(2)) < 1e-12


def test_launch_accounting_and_profile():
    """Launch counts per kernel class: a split above the one-CTA size runs the theta
    kernel once and one pivoted panel per 32 pivots; a small split is one launch."""
    from paper_2505_06119_gb300 import MPS

    rng = np.random.default_rng(1)
    with MPS(14, 64, precision="mixed", profile=True, policy="local") as m:
        m.set_site(6, states.complex_gaussian(rng, (64, 2, 64)).astype(np.complex64))
        m.set_site(7, states.complex_gaussian(rng, (64, 2, 64)).astype(np.complex64))
        m.apply_2q(6, gates.haar_unitary(rng, 4))
        m.sync()
        st = m.kernel_stats()
        assert st["theta"]["launches"] == 1
        assert st["panel"]["launches"] == 2  # k = 64 pivots, panel width 32
        assert st["panel"]["ms"] > 0
        m.kernel_stats_reset()
        assert m.kernel_stats()["panel"]["launches"] == 0
        m.apply_2q(0, gates.haar_unitary(rng, 4))  # theta 2 x 4: one CTA
        st = m.kernel_stats()
        assert st["panel"]["launches"] == 1 and st["theta"]["launches"] == 0


@pytest.mark.parametrize("noalloc", [False, True])
def test_raw_call_reports_expired_wait_as_nan(noalloc):
    """The raw-pointer calls have no handle: a bounded wait that expires shows as a
    NaN discarded weight; with the normal limits restored the next call is finite
    and correct (the error word and barrier words are cleared per call)."""
    import torch

    from paper_2505_06119_gb300 import _lib as L
    from paper_2505_06119_gb300.mps import _gate

    lib = L.load()
    rng = np.random.default_rng(5)
    cl, cm, cr, chi = 24, 16, 20, 32
    a = states.complex_gaussian(rng, (cl, 2, cm))
    b = states.complex_gaussian(rng, (cm, 2, cr))
    g = gates.haar_unitary(rng, 4)
    dev = torch.device("cuda:0")
    ta = torch.from_numpy(a).to(dev)
    tb = torch.from_numpy(b).to(dev)
    k = min(2 * cl, 2 * cr, chi)
    sz = ctypes.c_size_t()
    assert lib.mps_two_site_workspace(L.MPS_PREC_FP64, cl, cm, cr, chi, ctypes.byref(sz)) == 0
    ws = torch.empty(sz.value + 256, dtype=torch.uint8, device=dev)
    base = (ws.data_ptr() + 255) // 256 * 256
    stream = torch.cuda.current_stream().cuda_stream

    def call():
        oa = torch.empty((cl, 2, k), dtype=torch.complex128, device=dev)
        ob = torch.empty((k, 2, cr), dtype=torch.complex128, device=dev)
        disc = torch.zeros(1, dtype=torch.float64, device=dev)
        if noalloc:
            rc = lib.mps_two_site_apply_noalloc(L.MPS_PREC_FP64, cl, cm, cr, chi, ta.data_ptr(), tb.data_ptr(),
                                                _gate(g, 16), oa.data_ptr(), ob.data_ptr(), disc.data_ptr(), stream)
        else:
            rc = lib.mps_two_site_apply(L.MPS_PREC_FP64, cl, cm, cr, chi, ta.data_ptr(), tb.data_ptr(),
                                        _gate(g, 16), oa.data_ptr(), ob.data_ptr(), disc.data_ptr(), base,
                                        sz.value, stream)
        assert rc == 0
        torch.cuda.synchronize()
        return disc.item(), ob.cpu().numpy()

    assert lib.mps_debug_raw_wait(-1, 0.0) == L.MPS_E_ARG
    assert lib.mps_debug_raw_wait(1, 0.05) == 0
    try:
        d_bad, _ = call()
    finally:
        assert lib.mps_debug_raw_wait(0, 0.0) == 0
    assert np.isnan(d_bad)
    d_ok, ob = call()
    assert np.isfinite(d_ok) and d_ok > 0
    # kept norm + discarded weight = ||theta||^2 = ||A B||^2 (the gate is unitary)
    x = np.einsum("lcm,mdr->lcdr", a, b)
    assert d_ok + np.linalg.norm(ob) ** 2 == pytest.approx(np.linalg.norm(x) ** 2, rel=1e-10)


@pytest.mark.skipif("not __import__('torch').cuda.is_available() or __import__('torch').cuda.device_count() < 2",
                    reason="needs two visible GPUs")
def test_handles_and_raw_calls_on_two_devices():
    """First-use state (kernel attributes, occupancy) is kept per device: a handle on
    device 1 after one on device 0, and raw calls on both, all work."""
    import torch

    from paper_2505_06119_gb300 import MPS, _lib as L
    from paper_2505_06119_gb300.mps import _gate

    rng = np.random.default_rng(8)
    g = gates.haar_unitary(rng, 4)
    res = []
    for dev in (0, 1):
        with MPS(12, 64, precision="mixed", device=dev) as m:
            for i in range(11):
                m.apply_2q(i, g)
            m.move_centre(0)
            res.append(m.fidelity())
    assert res[0] == pytest.approx(res[1], rel=1e-6)
    lib = L.load()
    cl = cm = cr = chi = 48
    a = states.complex_gaussian(rng, (cl, 2, cm)).astype(np.complex64)
    b = states.complex_gaussian(rng, (cm, 2, cr)).astype(np.complex64)
    outs = []
    for dev in (0, 1):
        with torch.cuda.device(dev):
            d = torch.device("cuda:%d" % dev)
            ta, tb = torch.from_numpy(a).to(d), torch.from_numpy(b).to(d)
            oa = torch.empty((cl, 2, chi), dtype=torch.complex64, device=d)
            ob = torch.empty((chi, 2, cr), dtype=torch.complex64, device=d)
            disc = torch.zeros(1, dtype=torch.float64, device=d)
            rc = lib.mps_two_site_apply_noalloc(L.MPS_PREC_MIXED, cl, cm, cr, chi, ta.data_ptr(), tb.data_ptr(),
                                                _gate(g, 16), oa.data_ptr(), ob.data_ptr(), disc.data_ptr(),
                                                torch.cuda.current_stream().cuda_stream)
            assert rc == 0
            torch.cuda.synchronize()
            outs.append(ob.cpu().numpy())
    assert np.abs(outs[0] - outs[1]).max() <= 1e-6 * np.abs(outs[0]).max()
