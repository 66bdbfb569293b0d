"""Build the CUDA library ``_build/libmocd.so`` for sm_103a with nvcc.

Each translation unit is compiled in parallel, then linked into one shared
object exporting the C ABI of ``include/mocd.h``. Every source is built with
``-fmad=false`` so that no floating-point expression is contracted.
"""
from __future__ import annotations

import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "_build")
LIB = os.path.join(OUT, "libmocd.so")
SOURCES = ["k_eval.cu", "k_variation.cu", "k_select.cu", "runtime.cu", "noalloc.cu", "server.cu", "k_stats.cu", "k_graph.cu"]
HEADERS = ["mocd_internal.h", "philox.cuh", "mocd_check.cuh"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-fmad=false", "-Xcompiler", "-fPIC",
         "-I", os.path.join(ROOT, "include"), "-I", CSRC]


def _nvcc() -> str:
    home = os.environ.get("CUDA_HOME", "/usr/local/cuda")
    cand = os.path.join(home, "bin", "nvcc")
    return cand if os.path.exists(cand) else "nvcc"


def _stale(target: str, deps) -> bool:
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps)


OUT_DEBUG = os.path.join(HERE, "_build_debug")


def build(force: bool = False, verbose: bool = False, extra_flags=(), src_dir: str = CSRC,
          out_dir: str = None, debug: bool = False) -> str:
    """Compile ``src_dir`` into ``out_dir/libmocd.so``.

    Defaults: this package's sources into ``_build``. ``debug=True`` builds
    the variant whose kernels check their memory accesses' invariants and
    record failures instead of faulting (``-DMOCD_DEBUG_CHECKS``, into
    ``_build_debug``; see mocd_debug_checks). ``src_dir``, ``out_dir`` and
    ``extra_flags`` build a modified copy of the sources elsewhere, without
    touching this package's own library.
    """
    if out_dir is None:
        out_dir = OUT_DEBUG if debug else OUT
    if debug:
        extra_flags = tuple(extra_flags) + ("-DMOCD_DEBUG_CHECKS",)
    os.makedirs(out_dir, exist_ok=True)
    lib = os.path.join(out_dir, "libmocd.so")
    deps_common = [os.path.join(src_dir, h) for h in HEADERS] + [os.path.join(ROOT, "include", "mocd.h"),
                                                                 os.path.abspath(__file__)]
    nvcc = _nvcc()
    flags = [f if f != CSRC else src_dir for f in FLAGS]
    procs, objs = [], []
    for src in SOURCES:
        path = os.path.join(src_dir, src)
        obj = os.path.join(out_dir, src.replace(".cu", ".o"))
        objs.append(obj)
        if force or _stale(obj, [path] + deps_common):
            cmd = [nvcc, *ARCH, *flags, *extra_flags, "-c", path, "-o", obj]
            if verbose:
                print(" ".join(cmd), file=sys.stderr)
            procs.append((src, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)))
    failed = []
    for src, p in procs:
        out, _ = p.communicate()
        if out and (verbose or p.returncode):
            sys.stderr.write(out.decode())
        if p.returncode:
            failed.append(src)
    if failed:
        raise RuntimeError(f"nvcc failed for {failed}")
    if force or procs or _stale(lib, objs):
        tmp = lib + f".tmp{os.getpid()}"
        subprocess.run([nvcc, *ARCH, "-shared", "-o", tmp, *objs], check=True)
        os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
