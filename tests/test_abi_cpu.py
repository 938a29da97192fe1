"""CPU-side checks of the C ABI: the library builds, loads and exports every
function include/mps.h declares; host-side argument checks reject bad input
before any CUDA call.  No kernel is launched here."""

import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = []
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names += re.findall(r"^\s*(?:const\s+)?[A-Za-z_][\w\s\*]*?\b(mps_\w+)\s*\(", src, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    from paper_2505_06119_gb300 import build, _lib

    build.build()
    return _lib.load()


def test_header_declares_the_calls():
    names = declared_functions()
    for want in ["mps_create", "mps_apply_1q", "mps_apply_2q", "mps_swap", "mps_amplitude",
                 "mps_fidelity_estimate", "mps_destroy", "mps_apply_layer", "mps_overlap"]:
        assert want in names


def test_library_exports_every_declared_symbol(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name


@pytest.mark.parametrize("checked", [False, True])
def test_library_exports_only_the_c_abi(checked):
    """Both builds export the header's functions and no function-local static of the
    library's own code: a GNU-unique symbol (such a static of a template) would be one
    object for every build loaded into a process, so the second library would skip its
    own once-per-device setup (a kernel attribute) and its launch would fail."""
    import shutil
    import subprocess

    from paper_2505_06119_gb300 import build

    if not shutil.which("nm"):
        pytest.skip("nm not installed")
    path = build.build(checked=checked)
    out = subprocess.run(["nm", "-D", "--defined-only", path], capture_output=True, text=True, check=True).stdout
    syms = [line.split() for line in out.splitlines() if len(line.split()) == 3]
    assert not [s for s in syms if s[1] == "u"]
    text = {s[2] for s in syms if s[1] == "T"}
    assert text == set(declared_functions())


def test_binding_covers_every_declared_symbol():
    from paper_2505_06119_gb300 import _lib

    assert set(declared_functions()) <= set(_lib.SIGNATURES)


def test_binding_arity_matches_the_header():
    """Every prototype in include/*.h has a binding signature with the same number of
    parameters, so a ctypes call can never shift its arguments."""
    from paper_2505_06119_gb300 import _lib

    for fn in os.listdir(os.path.join(ROOT, "include")):
        if not fn.endswith(".h"):
            continue
        src = re.sub(r"/\*.*?\*/", "", open(os.path.join(ROOT, "include", fn)).read(), flags=re.S)
        protos = re.findall(r"^\s*(?:const\s+)?[A-Za-z_][\w\s\*]*?\b(mps_\w+)\s*\(([^)]*)\)\s*;", src, flags=re.M)
        assert protos
        for name, args in protos:
            args = args.strip()
            n = 0 if args in ("", "void") else len([a for a in args.split(",") if a.strip()])
            assert len(_lib.SIGNATURES[name][1]) == n, name


def test_host_argument_checks(lib):
    from paper_2505_06119_gb300 import _lib as L

    h = ctypes.c_void_p()
    assert lib.mps_create(ctypes.byref(h), 0, 4) == L.MPS_E_ARG
    assert lib.mps_create(ctypes.byref(h), 4, 0) == L.MPS_E_ARG
    assert lib.mps_create(None, 4, 4) == L.MPS_E_ARG
    cfg = L.mps_config()
    lib.mps_config_init(ctypes.byref(cfg))
    assert cfg.precision == L.MPS_PREC_FP64 and cfg.policy == L.MPS_POLICY_CANON
    cfg.precision = 7
    assert lib.mps_create_ex(ctypes.byref(h), 4, 4, ctypes.byref(cfg)) == L.MPS_E_ARG
    lib.mps_config_init(ctypes.byref(cfg))
    cfg.panel_width = 33
    assert lib.mps_create_ex(ctypes.byref(h), 4, 4, ctypes.byref(cfg)) == L.MPS_E_ARG
    lib.mps_config_init(ctypes.byref(cfg))
    cfg.debug_max_ctas = -1
    assert lib.mps_create_ex(ctypes.byref(h), 4, 4, ctypes.byref(cfg)) == L.MPS_E_ARG
    lib.mps_config_init(ctypes.byref(cfg))
    cfg.debug_barrier_extra = -1
    assert lib.mps_create_ex(ctypes.byref(h), 4, 4, ctypes.byref(cfg)) == L.MPS_E_ARG
    lib.mps_config_init(ctypes.byref(cfg))
    assert cfg.truncation == L.MPS_TRUNC_QRCP
    cfg.truncation = 3  # unknown truncation mode
    assert lib.mps_create_ex(ctypes.byref(h), 4, 4, ctypes.byref(cfg)) == L.MPS_E_ARG
    cfg.truncation = L.MPS_TRUNC_SVD  # the SVD split is limited to chi_max <= 4096
    assert lib.mps_create_ex(ctypes.byref(h), 30, 8192, ctypes.byref(cfg)) == L.MPS_E_UNSUPPORTED
    assert lib.mps_destroy(None) == L.MPS_OK
    assert lib.mps_apply_2q(None, 0, None, 4) == L.MPS_E_ARG
    assert lib.mps_version() >= 100


def test_workspace_query_is_host_only(lib):
    from paper_2505_06119_gb300 import _lib as L

    sz = ctypes.c_size_t()
    assert lib.mps_two_site_workspace(L.MPS_PREC_FP64, 64, 64, 64, 64, ctypes.byref(sz)) == L.MPS_OK
    small = sz.value
    assert lib.mps_two_site_workspace(L.MPS_PREC_FP64, 128, 128, 128, 128, ctypes.byref(sz)) == L.MPS_OK
    assert sz.value > small
    assert lib.mps_two_site_workspace(L.MPS_PREC_MIXED, 128, 128, 128, 128, ctypes.byref(sz)) == L.MPS_OK
    assert lib.mps_two_site_workspace(L.MPS_PREC_FP64, 0, 1, 1, 1, ctypes.byref(sz)) == L.MPS_E_ARG


@pytest.mark.parametrize("lang", ["c", "c++"])
def test_header_compiles_as_c_and_cpp(lang, tmp_path):
    """include/mps.h is a plain C header usable from C and C++ callers."""
    import shutil
    import subprocess

    cc = shutil.which("gcc" if lang == "c" else "g++")
    if cc is None:
        pytest.skip("no host compiler")
    src = tmp_path / ("use.c" if lang == "c" else "use.cpp")
    src.write_text('#include "mps.h"\nint main(void) { mps_config c; mps_config_init(&c); return c.precision; }\n')
    r = subprocess.run([cc, "-x", lang, "-fsyntax-only", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"),
                        str(src)], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
