"""Builds libdibella.so in-tree with nvcc for sm_103a (no torch extension machinery)."""

from __future__ import annotations

import os
import subprocess
import threading

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
LIB = os.path.join(HERE, "libdibella.so")
# The same library with every kernel bounds check compiled in (DIBELLA_BOUNDS_CHECK).
LIB_DEBUG = os.path.join(HERE, "libdibella_debug.so")
SOURCES = [os.path.join(CSRC, "dibella_xdrop.cu"), os.path.join(CSRC, "dibella_kmers.cu"),
           os.path.join(CSRC, "dibella_traceback.cu"), os.path.join(CSRC, "dibella_peak.cu"),
           os.path.join(CSRC, "dibella_pack.cpp")]
HEADERS = [os.path.join(INCLUDE, "dibella.h")]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
_lock = threading.Lock()


def _nvcc() -> str:
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if cand and (os.path.sep not in cand or os.path.exists(cand)):
            return cand
    return "nvcc"


def _stale(target: str, deps) -> bool:
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps)


def lib_path(debug: bool = False) -> str:
    return LIB_DEBUG if debug else LIB


def build(force: bool = False, verbose: bool = False, debug: bool = False) -> str:
    """Compile every translation unit in parallel and link libdibella.so (or,
    with debug, libdibella_debug.so with the kernels' bounds checks)."""
    target = lib_path(debug)
    with _lock:
        if not force and not _stale(target, SOURCES + HEADERS + [__file__]):
            return target
        objs, procs = [], []
        for src in SOURCES:
            obj = os.path.join(CSRC, os.path.basename(src) + (".dbg.o" if debug else ".o"))
            cmd = [_nvcc(), *ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC",
                   "-Xcompiler", "-pthread", "-I", INCLUDE, "-c", src, "-o", obj]
            if debug:
                cmd.insert(1, "-DDIBELLA_BOUNDS_CHECK")
            if src.endswith(".cu"):
                cmd[1:1] = ["-Xptxas", "-v"] if verbose else []
            procs.append(subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT))
            objs.append(obj)
        for p, src in zip(procs, SOURCES):
            out, _ = p.communicate()
            if p.returncode != 0:
                raise RuntimeError("nvcc failed on %s:\n%s" % (src, out.decode(errors="replace")))
            if verbose and out:
                print(out.decode(errors="replace"))
        tmp = target + ".tmp%d" % os.getpid()
        subprocess.check_call([_nvcc(), *ARCH, "-shared", "-cudart", "static", "-o", tmp, *objs, "-lpthread"])
        os.replace(tmp, target)
        for o in objs:
            os.remove(o)
    return target
