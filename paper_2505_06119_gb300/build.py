"""Build the CUDA library in-tree: paper_2505_06119_gb300/_build/libmps_gb300.so.

Each .cu file is compiled for sm_103a only (GB300) in parallel, then linked
as a shared library with a plain C ABI (include/mps.h).  Rebuilds only what
changed.
"""

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
SRC_DIR = os.path.join(HERE, "csrc")
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(OUT_DIR, "libmps_gb300.so")
# the bounds-checking variant (-DMPS_BOUNDS_CHECK): kernels verify indices taken from
# device data and report DEV_ERR_BOUNDS instead of accessing out of range
CHECKED_DIR = os.path.join(HERE, "_build_checked")
CHECKED_LIB = os.path.join(CHECKED_DIR, "libmps_gb300_checked.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc():
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", shutil.which("nvcc")):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build the library")


def sources():
    return sorted(os.path.join(SRC_DIR, f) for f in os.listdir(SRC_DIR) if f.endswith(".cu"))


def headers():
    hs = [os.path.join(SRC_DIR, f) for f in os.listdir(SRC_DIR) if f.endswith((".h", ".cuh"))]
    hs.append(os.path.join(ROOT, "include", "mps.h"))
    return hs


def _compile(src, obj, extra):
    # hidden visibility: only the C ABI of include/mps.h is exported, so two builds
    # loaded into one process (the checked and the plain library) share no symbol
    # (function-local statics of templates would otherwise be unified across them)
    cmd = [nvcc(), *ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC,-fvisibility=hidden",
           "-I", os.path.join(ROOT, "include"), *extra, "-c", src, "-o", obj]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("nvcc failed for %s:\n%s\n%s" % (src, r.stdout, r.stderr))
    return r.stderr


def build(force=False, verbose=False, extra=(), checked=False):
    """Build the library (checked=True: the bounds-checking variant) and return its path."""
    out_dir = CHECKED_DIR if checked else OUT_DIR
    lib = CHECKED_LIB if checked else LIB
    extra = list(extra) + (["-DMPS_BOUNDS_CHECK"] if checked else [])
    os.makedirs(out_dir, exist_ok=True)
    hdr_time = max(os.path.getmtime(h) for h in headers())
    objs, todo = [], []
    for src in sources():
        obj = os.path.join(out_dir, os.path.basename(src)[:-3] + ".o")
        objs.append(obj)
        if force or not os.path.exists(obj) or os.path.getmtime(obj) < max(os.path.getmtime(src), hdr_time):
            todo.append((src, obj))
    if todo:
        with cf.ThreadPoolExecutor(max_workers=min(8, len(todo))) as ex:
            futs = {ex.submit(_compile, s, o, list(extra)): s for s, o in todo}
            for f in cf.as_completed(futs):
                msg = f.result()
                if verbose and msg:
                    print(futs[f], msg, file=sys.stderr)
    if todo or not os.path.exists(lib):
        tmp = lib + ".tmp.%d" % os.getpid()
        cmd = [nvcc(), *ARCH, "-shared", "-o", tmp, *objs, "-lcudart"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("link failed:\n%s\n%s" % (r.stdout, r.stderr))
        os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    force = "--force" in sys.argv
    extra = ["-Xptxas", "-v"] if "--ptxas" in sys.argv else []
    print(build(force=force, verbose=True, extra=extra, checked="--checked" in sys.argv))
