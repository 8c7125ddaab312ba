"""In-tree build of the CUDA library (sm_103a only) with nvcc.

Every ``csrc/*.cu`` file is compiled to an object in ``_build/`` in parallel,
then linked into ``_lib/libmbs_gb300.so``. Objects are rebuilt when their source
or any header is newer. ``bounds_check=True`` builds the index-checking variant
(``-DMBS_BOUNDS_CHECK``) into ``_build_checked/`` and
``_lib/libmbs_gb300_checked.so``.
"""
from __future__ import annotations

import concurrent.futures as cf
import glob
import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIBDIR = os.path.join(HERE, "_lib")
LIB = os.path.join(LIBDIR, "libmbs_gb300.so")
LIB_CHECKED = os.path.join(LIBDIR, "libmbs_gb300_checked.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-std=c++17", "-O3", "-lineinfo", "-Xcompiler", "-fPIC", "-Xcompiler", "-fvisibility=hidden",
         "-I" + os.path.join(ROOT, "include")]


def _nvcc():
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build the library")


def _headers():
    return glob.glob(os.path.join(CSRC, "*.cuh")) + glob.glob(os.path.join(CSRC, "*.h")) + \
        glob.glob(os.path.join(ROOT, "include", "*.h"))


def _stale(obj, src, hdr_mtime):
    if not os.path.exists(obj):
        return True
    m = os.path.getmtime(obj)
    return os.path.getmtime(src) > m or hdr_mtime > m


def build(verbose=False, jobs=None, bounds_check=False):
    """Compile and link the library; returns the path of the shared object."""
    nvcc = _nvcc()
    build_dir = BUILD + "_checked" if bounds_check else BUILD
    lib = LIB_CHECKED if bounds_check else LIB
    flags = FLAGS + (["-DMBS_BOUNDS_CHECK"] if bounds_check else [])
    os.makedirs(build_dir, exist_ok=True)
    os.makedirs(LIBDIR, exist_ok=True)
    srcs = sorted(glob.glob(os.path.join(CSRC, "*.cu")))
    hdr_mtime = max([os.path.getmtime(h) for h in _headers()] + [0.0])
    objs = []
    todo = []
    for s in srcs:
        o = os.path.join(build_dir, os.path.splitext(os.path.basename(s))[0] + ".o")
        objs.append(o)
        if _stale(o, s, hdr_mtime):
            todo.append((s, o))

    def compile_one(so):
        s, o = so
        cmd = [nvcc] + ARCH + flags + ["-c", s, "-o", o]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("nvcc failed for %s:\n%s\n%s" % (s, r.stdout, r.stderr))
        if verbose:
            print("built", os.path.basename(o), flush=True)

    # largest translation units first
    todo.sort(key=lambda so: -os.path.getsize(so[0]))
    nj = jobs or max(1, min(len(todo), os.cpu_count() or 4))
    if todo:
        with cf.ThreadPoolExecutor(max_workers=nj) as ex:
            list(ex.map(compile_one, todo))
    if todo or not os.path.exists(lib):
        cmd = [nvcc] + ARCH + ["-shared", "-o", lib + ".tmp"] + objs
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("link failed:\n%s\n%s" % (r.stdout, r.stderr))
        os.replace(lib + ".tmp", lib)
    return lib


if __name__ == "__main__":
    import time

    t = time.time()
    print(build(verbose=True), "%.1fs" % (time.time() - t))
