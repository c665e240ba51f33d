"""Build the ggeval CUDA library in-tree: csrc/*.cu -> _lib/libggeval.so.

Each translation unit is compiled by nvcc for sm_103a in parallel, then
linked into one shared library (CUDA runtime linked statically).  Objects
go to ``_build/`` next to this file; both folders are git-ignored.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
OUT = os.path.join(HERE, "_lib", "libggeval.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
GEN = os.path.join(BUILD, "gen")  # generated sources (the PTX interpreter)
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr",
         "-I", os.path.join(ROOT, "include"), "-I", CSRC, "-I", GEN]


def _nvcc():
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def sources():
    return sorted(f for f in os.listdir(CSRC) if f.endswith(".cu"))


def _stale(obj, deps):
    if not os.path.exists(obj):
        return True
    t = os.path.getmtime(obj)
    return any(os.path.getmtime(d) > t for d in deps)


def build(verbose: bool = False, extra_flags=(), force: bool = False, out: str = OUT,
          build_dir: str = BUILD) -> str:
    """Compile every csrc/*.cu for sm_103a and link the library.  A variant
    build (extra compiler flags) takes its own `out` and `build_dir`."""
    nvcc = _nvcc()
    os.makedirs(build_dir, exist_ok=True)
    os.makedirs(os.path.dirname(out), exist_ok=True)
    # the interpreter's inline PTX, written only when its text changes
    sys.path.insert(0, CSRC)
    try:
        import interp_gen
    finally:
        sys.path.pop(0)
    gen_inc = os.path.join(GEN, "interp_asm.inc")
    interp_gen.main(gen_inc)
    headers = [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".h", ".cuh"))]
    headers += [os.path.join(ROOT, "include", "ggeval.h"), gen_inc]
    jobs = []
    objs = []
    for src in sources():
        s = os.path.join(CSRC, src)
        o = os.path.join(build_dir, src[:-3] + ".o")
        objs.append(o)
        if force or _stale(o, [s, *headers, __file__]):
            jobs.append([nvcc, *ARCH, *FLAGS, *extra_flags, "-c", s, "-o", o])

    def run(cmd):
        r = subprocess.run(cmd, capture_output=True, text=True)
        return cmd, r

    with cf.ThreadPoolExecutor(max_workers=max(1, min(len(jobs), os.cpu_count() or 4))) as ex:
        for cmd, r in ex.map(run, jobs):
            if verbose or r.returncode:
                sys.stderr.write(" ".join(cmd) + "\n" + r.stdout + r.stderr)
            if r.returncode:
                raise RuntimeError(f"nvcc failed on {cmd[-3]}")
    if force or jobs or not os.path.exists(out) or _stale(out, objs):
        cmd = [nvcc, *ARCH, "-shared", "-o", out, *objs, "-cudart", "static"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode:
            sys.stderr.write(" ".join(cmd) + "\n" + r.stdout + r.stderr)
            raise RuntimeError("link failed")
    return out


CHECKED_OUT = os.path.join(HERE, "_lib", "libggeval_checked.so")
CHECKED_BUILD = os.path.join(HERE, "_build_checked")


def build_checked(verbose: bool = False, force: bool = False) -> str:
    """The checked library: the C++ interpreter with every shared-memory
    stack and feature access and every tile copy bounds-checked
    (GGEVAL_CHECKED; a violation is recorded in the status word, never
    trapped).  For tests on small cases."""
    return build(verbose, ["-DGGEVAL_CHECKED", "-DGG_INTERP_CXX"], force, CHECKED_OUT,
                 CHECKED_BUILD)


def build_all(verbose: bool = False, force: bool = False):
    """The library and its checked build, compiled side by side."""
    with cf.ThreadPoolExecutor(max_workers=2) as ex:
        a = ex.submit(build, verbose, (), force)
        b = ex.submit(build_checked, verbose, force)
        return a.result(), b.result()


if __name__ == "__main__":
    print(build_all(verbose="-v" in sys.argv, force="-f" in sys.argv))
