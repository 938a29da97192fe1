"""Thin Python binding of the C ABI: one class per handle, argument marshalling only.

Every operation runs in the CUDA library (include/mps.h); this module only
converts NumPy arrays to the ABI's plain arrays and checks return codes.
"""

import ctypes

import numpy as np

from . import _lib as L


class MPSError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("%s (%d): %s" % (L.ERROR_NAMES.get(code, "?"), code, msg))
        self.code = code


def _gate(g, n):
    g = np.ascontiguousarray(np.asarray(g, dtype=np.complex128).reshape(-1))
    if g.size != n:
        raise ValueError("gate must have %d entries" % n)
    arr = (L.mps_c128 * n)()
    for i in range(n):
        arr[i].re = g[i].real
        arr[i].im = g[i].imag
    return arr


def config(precision="fp64", policy="canon", panel_width=0, stream=None, profile=False,
           wait_timeout_s=0.0, device=0, debug_barrier_extra=0, tensor_cores=False, debug_max_ctas=0,
           truncation="qrcp", sketch_seed=0, autotune=False, graphs=True):
    lib = L.load()
    cfg = L.mps_config()
    lib.mps_config_init(ctypes.byref(cfg))
    cfg.precision = {"fp64": L.MPS_PREC_FP64, "mixed": L.MPS_PREC_MIXED}[precision]
    cfg.policy = {"canon": L.MPS_POLICY_CANON, "local": L.MPS_POLICY_LOCAL}[policy]
    cfg.panel_width = panel_width
    cfg.stream = stream
    cfg.flags = ((L.MPS_FLAG_PROFILE if profile else 0) | (L.MPS_FLAG_TENSOR_CORES if tensor_cores else 0)
                 | (L.MPS_FLAG_AUTOTUNE if autotune else 0) | (0 if graphs else L.MPS_FLAG_NO_GRAPH))
    cfg.wait_timeout_s = wait_timeout_s
    cfg.device = device
    cfg.debug_barrier_extra = debug_barrier_extra
    cfg.debug_max_ctas = debug_max_ctas
    cfg.truncation = {"qrcp": L.MPS_TRUNC_QRCP, "svd": L.MPS_TRUNC_SVD, "rqrcp": L.MPS_TRUNC_RQRCP}[truncation]
    cfg.sketch_seed = sketch_seed
    return cfg


class MPS:
    """An n-qubit MPS on the GPU (handle of the C library)."""

    def __init__(self, n, chi_max, precision="fp64", policy="canon", lib=None, **kw):
        self.lib = lib if lib is not None else L.load()
        self.n = n
        self.chi_max = chi_max
        self.precision = precision
        self.policy = policy
        cfg = config(precision, policy, **kw)
        h = ctypes.c_void_p()
        rc = self.lib.mps_create_ex(ctypes.byref(h), n, chi_max, ctypes.byref(cfg))
        if rc != L.MPS_OK:
            raise MPSError(rc, "mps_create_ex failed")
        self.h = h

    def _check(self, rc):
        if rc != L.MPS_OK:
            msg = self.lib.mps_last_error(self.h)
            raise MPSError(rc, msg.decode() if msg else "")
        return rc

    def close(self):
        if getattr(self, "h", None):
            self.lib.mps_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    # ---- gates
    def apply_1q(self, q, u):
        self._check(self.lib.mps_apply_1q(self.h, q, _gate(u, 4)))

    def apply_2q(self, i, g, chi_max=0):
        self._check(self.lib.mps_apply_2q(self.h, i, _gate(g, 16), chi_max))

    def swap(self, i, chi_max=0):
        self._check(self.lib.mps_swap(self.h, i, chi_max))

    def apply_2q_routed(self, q1, q2, g, chi_max=0):
        self._check(self.lib.mps_apply_2q_routed(self.h, q1, q2, _gate(g, 16), chi_max))

    def apply_layer(self, sites, gates, chi_max=0):
        cnt = len(sites)
        s = (ctypes.c_int * max(cnt, 1))(*sites)
        g = _gate(np.concatenate([np.asarray(x).reshape(-1) for x in gates]) if cnt else np.zeros(16), 16 * max(cnt, 1))
        self._check(self.lib.mps_apply_layer(self.h, s, g, cnt, chi_max))

    def apply_mpo(self, first, ws, chi_max=0):
        """MPO (list of W[a, b, out, in] arrays) on sites first .. first+len(ws)-1."""
        ws = [np.asarray(x, dtype=np.complex128) for x in ws]
        bonds = [w.shape[0] for w in ws] + [ws[-1].shape[1]]
        flat = np.concatenate([np.ascontiguousarray(w).reshape(-1) for w in ws])
        b = (ctypes.c_int * len(bonds))(*bonds)
        self._check(self.lib.mps_apply_mpo(self.h, first, len(ws), b, _gate(flat, flat.size), chi_max))

    def permute(self, order, chi_max=0):
        """Site permutation by bubble-sorted SWAPs: position p ends up holding the site
        now at order[p].  Returns the number of SWAPs."""
        o = (ctypes.c_int * max(len(order), 1))(*[int(x) for x in order])
        cnt = ctypes.c_longlong()
        self._check(self.lib.mps_permute(self.h, o, chi_max, ctypes.byref(cnt)))
        return cnt.value

    def permute_layers(self, order, chi_max=0):
        """The same permutation by odd-even transposition sort, one layer of disjoint
        SWAPs per pass (local policy).  Returns (SWAPs, passes)."""
        o = (ctypes.c_int * max(len(order), 1))(*[int(x) for x in order])
        cnt = ctypes.c_longlong()
        npass = ctypes.c_int()
        self._check(self.lib.mps_permute_layers(self.h, o, chi_max, ctypes.byref(cnt), ctypes.byref(npass)))
        return cnt.value, npass.value

    def run(self, ops, chi_max=0):
        for op in ops:
            if op[0] == "1q":
                self.apply_1q(op[1], op[2])
            elif op[0] == "perm":
                self.permute(op[1], chi_max)
            elif op[0] == "mpo":
                self.apply_mpo(op[1], op[2], chi_max)
            elif abs(op[1] - op[2]) == 1 and op[1] < op[2]:
                self.apply_2q(op[1], op[3], chi_max)
            else:
                self.apply_2q_routed(op[1], op[2], op[3], chi_max)

    # ---- observables
    def amplitude(self, bits):
        b = (ctypes.c_uint8 * self.n)(*[int(x) for x in bits])
        out = L.mps_c128()
        self._check(self.lib.mps_amplitude(self.h, b, ctypes.byref(out)))
        return complex(out.re, out.im)

    def fidelity(self):
        out = ctypes.c_double()
        self._check(self.lib.mps_fidelity_estimate(self.h, ctypes.byref(out)))
        return out.value

    def overlap(self, other):
        out = L.mps_c128()
        self._check(self.lib.mps_overlap(self.h, other.h, ctypes.byref(out)))
        return complex(out.re, out.im)

    def bond_dims(self):
        arr = (ctypes.c_int * (self.n + 1))()
        self._check(self.lib.mps_bond_dims(self.h, arr))
        return list(arr)

    def get_site(self, i, fmt="c128", out=None):
        b = self.bond_dims()
        shape = (b[i], 2, b[i + 1])
        dt = np.complex128 if fmt == "c128" else np.complex64
        if out is None:
            out = np.empty(shape, dtype=dt)
        elif out.shape != shape or out.dtype != dt or not out.flags.c_contiguous:
            raise ValueError("out must be a contiguous %s array of shape %s" % (dt, shape))
        code = L.MPS_HOST_C128 if fmt == "c128" else L.MPS_HOST_C64
        self._check(self.lib.mps_get_site(self.h, i, code, out.ctypes.data, out.size))
        return out

    def set_site(self, i, a):
        a = np.asarray(a)
        if a.dtype == np.complex64:
            code = L.MPS_HOST_C64
        else:
            a = a.astype(np.complex128)
            code = L.MPS_HOST_C128
        a = np.ascontiguousarray(a)
        self._check(self.lib.mps_set_site(self.h, i, a.shape[0], a.shape[2], code, a.ctypes.data))

    def set_sites(self, sites, centre=0):
        for i, s in enumerate(sites):
            self.set_site(i, s)
        self._check(self.lib.mps_set_centre(self.h, centre))

    def set_centre(self, centre):
        self._check(self.lib.mps_set_centre(self.h, centre))

    def centre(self):
        c = ctypes.c_int()
        self._check(self.lib.mps_get_centre(self.h, ctypes.byref(c)))
        return c.value

    def move_centre(self, target):
        self._check(self.lib.mps_move_centre(self.h, target))

    def discarded(self):
        t = ctypes.c_double()
        c = ctypes.c_longlong()
        self._check(self.lib.mps_discarded_weight(self.h, ctypes.byref(t), ctypes.byref(c)))
        return t.value, c.value

    def svd_stats(self):
        """(sweeps, rotations) of the most recent SVD split (truncation="svd" handles)."""
        sw = ctypes.c_int()
        rot = ctypes.c_longlong()
        self._check(self.lib.mps_svd_last_stats(self.h, ctypes.byref(sw), ctypes.byref(rot)))
        return sw.value, rot.value

    def last_pivots(self):
        """(jpvt, k) of the most recent pivoted two-site split: jpvt[t] is the theta
        column (b * chi_r + r) at pivot position t; the first k were kept."""
        b = self.bond_dims()
        cap = 2 * max(b) + 2
        arr = (ctypes.c_int * cap)()
        n = ctypes.c_int()
        k = ctypes.c_int()
        self._check(self.lib.mps_last_split_pivots(self.h, arr, cap, ctypes.byref(n), ctypes.byref(k)))
        return np.array(arr[:n.value], dtype=np.int64), k.value

    def sync(self):
        self._check(self.lib.mps_sync(self.h))

    def set_stream(self, stream_ptr):
        self._check(self.lib.mps_set_stream(self.h, stream_ptr))

    def kernel_stats(self):
        arr = (L.mps_kstat * L.KCLASS_COUNT)()
        self._check(self.lib.mps_kernel_stats(self.h, arr))
        return {name: {"launches": arr[i].launches, "ms": arr[i].ms, "alg_bytes": arr[i].alg_bytes,
                       "alg_flops": arr[i].alg_flops} for i, name in enumerate(L.KCLASS)}

    def layer_stats(self):
        """(layer calls, of them run as a CUDA graph launch, graphs still on)."""
        a, b, c = ctypes.c_longlong(), ctypes.c_longlong(), ctypes.c_int()
        self._check(self.lib.mps_layer_stats(self.h, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)))
        return a.value, b.value, bool(c.value)

    def kernel_stats_reset(self):
        self._check(self.lib.mps_kernel_stats_reset(self.h))


def tune_two_site(precision, chi_l, chi_m, chi_r, chi_max, force=False):
    """Autotune one two-site split shape (mps_tune_two_site): returns a dict with the
    chosen panel width and panel CTA count, the candidates timed and the times."""
    lib = L.load()
    out = L.mps_tune_result()
    code = {"fp64": L.MPS_PREC_FP64, "mixed": L.MPS_PREC_MIXED}[precision]
    rc = lib.mps_tune_two_site(code, chi_l, chi_m, chi_r, chi_max, 1 if force else 0, ctypes.byref(out))
    if rc != 0:
        raise MPSError(rc, "mps_tune_two_site failed")
    return {"panel_width": out.panel_width, "panel_ctas": out.panel_ctas, "candidates": out.candidates,
            "ms": out.ms, "default_ms": out.default_ms}
