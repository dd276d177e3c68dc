"""Builds the CUDA library libphmm.so in-tree (paper_2606_25738_gb300/_lib/) with nvcc
for sm_103a: the translation units compiled in parallel, then linked as a shared
library exporting the C ABI of include/phmm.h.  build_cpu() builds the separate host
comparator libphmm_cpu.so (include/phmm_cpu.h) with the C compiler."""
from __future__ import annotations

import os
import shutil
import subprocess
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
LIBDIR = os.path.join(HERE, "_lib")
LIB = os.path.join(LIBDIR, "libphmm.so")
SOURCES = ["kernels_f32.cu", "kernels_f64.cu", "runtime.cu", "noalloc.cu", "serve.cpp"]
CPU_SOURCE = "cpu_rowwise.c"
CPU_DEPS = ["cpu_rowwise.c", "cpu_engine.inc"]
CPU_LIB = os.path.join(LIBDIR, "libphmm_cpu.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2",
         "-diag-suppress", "177", "-I" + os.path.join(ROOT, "include"), "-I" + CSRC]


def nvcc() -> str:
    p = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(p):
        raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libphmm")
    return p


def _stale() -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    deps = [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f not in CPU_DEPS] + [
        os.path.join(ROOT, "include", "phmm.h"), os.path.abspath(__file__)]
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False) -> str:
    """Compile (if sources changed) and return the path of libphmm.so."""
    if not force and not _stale():
        return LIB
    os.makedirs(LIBDIR, exist_ok=True)
    nv = nvcc()
    tag = str(os.getpid())

    def compile_one(src: str) -> str:
        obj = os.path.join(LIBDIR, os.path.splitext(src)[0] + ".%s.o" % tag)
        cmd = [nv, *ARCH, *FLAGS, "-c", os.path.join(CSRC, src), "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("nvcc failed for %s:\n%s" % (src, r.stderr[-4000:]))
        if verbose and r.stderr:
            print(r.stderr)
        return obj

    with ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        objs = list(ex.map(compile_one, SOURCES))
    tmp = LIB + "." + tag
    r = subprocess.run([nv, *ARCH, "-shared", "-o", tmp, *objs], capture_output=True, text=True)
    for o in objs:
        os.remove(o)
    if r.returncode != 0:
        raise RuntimeError("link failed:\n" + r.stderr[-4000:])
    os.replace(tmp, LIB)
    return LIB


def build_cpu(force: bool = False) -> str:
    """Compile (if its sources changed) and return the path of libphmm_cpu.so.  Portable
    flags only (-O3, no -march: the generic vector types map to the host's baseline SIMD,
    NEON on Arm and SSE2 on x86); FMA contraction is allowed where the host has FMA."""
    src = os.path.join(CSRC, CPU_SOURCE)
    deps = [os.path.join(CSRC, f) for f in CPU_DEPS] + [
        os.path.join(ROOT, "include", "phmm_cpu.h"), os.path.join(ROOT, "include", "phmm.h"),
        os.path.abspath(__file__)]
    if not force and os.path.exists(CPU_LIB) and all(os.path.getmtime(d) <= os.path.getmtime(CPU_LIB) for d in deps):
        return CPU_LIB
    os.makedirs(LIBDIR, exist_ok=True)
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        raise RuntimeError("no C compiler for libphmm_cpu.so")
    tmp = CPU_LIB + "." + str(os.getpid())
    r = subprocess.run([cc, "-O3", "-std=gnu11", "-ffp-contract=fast", "-fPIC", "-shared", "-pthread",
                        "-I" + os.path.join(ROOT, "include"),
                        src, "-o", tmp, "-lm"], capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("cc failed for %s:\n%s" % (CPU_SOURCE, r.stderr[-4000:]))
    os.replace(tmp, CPU_LIB)
    return CPU_LIB


if __name__ == "__main__":
    print(build(force=True, verbose=True))
    print(build_cpu(force=True))
