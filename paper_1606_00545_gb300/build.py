"""Build the CUDA library ``_build/libhecgpu.so`` for sm_103a with nvcc.

Each translation unit is compiled in parallel (one ``-gencode``), then linked
into one shared library with the CUDA runtime linked statically.  Object files
are rebuilt when a source or header is newer than the library.  ``debug=True``
builds the same sources with ``-DHEC_DEBUG`` (device-side checks) into
``_build/debug/libhecgpu.so``.
"""
from __future__ import annotations

import fcntl
import glob
import os
import subprocess
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "_build")
LIB = os.path.join(OUT, "libhecgpu.so")
GENCODE = "arch=compute_103a,code=sm_103a"


def _nvcc() -> str:
    cand = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "bin", "nvcc")
    return cand if os.path.exists(cand) else "nvcc"


def sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")) + glob.glob(os.path.join(CSRC, "*.cpp")))


def _deps():
    return sources() + glob.glob(os.path.join(CSRC, "*.h")) + glob.glob(
        os.path.join(CSRC, "*.cuh")) + [os.path.join(ROOT, "include", "hecgpu.h"), __file__]


def _paths(debug: bool):
    out = os.path.join(OUT, "debug") if debug else OUT
    return out, os.path.join(out, "libhecgpu.so")


def _current(lib: str) -> bool:
    if not os.path.exists(lib):
        return False
    t = os.path.getmtime(lib)
    return all(os.path.getmtime(d) <= t for d in _deps())


def build(force: bool = False, verbose: bool = False, debug: bool = False) -> str:
    """Compile and link the library if anything changed; return its path.
    Processes that build at the same time (the ranks of one launch, parallel
    test workers) take turns on a lock file: one compiles, the others then
    find the library current."""
    out, lib = _paths(debug)
    os.makedirs(out, exist_ok=True)
    if not force and _current(lib):
        return lib
    with open(os.path.join(out, ".build.lock"), "w") as lock:
        fcntl.flock(lock, fcntl.LOCK_EX)
        if not force and _current(lib):
            return lib
        return _compile(verbose, debug)


def _compile(verbose: bool, debug: bool = False) -> str:
    out, lib = _paths(debug)
    nvcc = _nvcc()
    common = ["-gencode", GENCODE, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC",
              "-Xcompiler", "-ffp-contract=off", "-I", os.path.join(ROOT, "include")]
    if debug:
        common.append("-DHEC_DEBUG")

    def compile_one(src):
        obj = os.path.join(out, os.path.basename(src) + ".o")
        cmd = [nvcc] + common + ["-c", src, "-o", obj]
        if src.endswith(".cpp"):
            cmd[1:1] = ["-x", "c++"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("nvcc failed for %s:\n%s\n%s" % (src, r.stdout, r.stderr))
        if verbose and (r.stdout or r.stderr):
            print(r.stdout, r.stderr)
        return obj

    with ThreadPoolExecutor(max_workers=min(8, os.cpu_count() or 1)) as ex:
        objs = list(ex.map(compile_one, sources()))
    tmp = lib + ".%d.tmp" % os.getpid()
    cmd = [nvcc, "-gencode", GENCODE, "-shared", "-o", tmp] + objs + ["-lpthread"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("link failed:\n%s\n%s" % (r.stdout, r.stderr))
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    print(build(force=True, verbose=True))
