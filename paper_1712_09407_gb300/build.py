"""In-tree build of libtpcca.so (the CUDA tracker behind include/tpcca.h) for sm_103a.

Each .cu file is compiled in parallel with nvcc, then linked as a shared library next to
this file.  Floating-point contraction is off on both the device (-fmad=false) and the host
side, so every expression rounds exactly as written.
"""
from __future__ import annotations

import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libtpcca.so")
# The checked build: the same library with every data-dependent pool index checked in the kernels
# (-DTPC_CHECKED); a failed check reports TPC_ERR_CHECK.  The tests run it next to the release one.
BUILD_CHECKED = os.path.join(HERE, "_build_checked")
LIB_CHECKED = os.path.join(HERE, "libtpcca_checked.so")
SOURCES = ["api.cu", "k_links.cu", "k_construct.cu", "k_sweep.cu", "k_select.cu", "k_global.cu", "k_merge.cu", "noalloc.cu", "server.cu"]
HEADERS = [os.path.join(CSRC, "common.cuh"), os.path.join(CSRC, "kf.cuh"), os.path.join(os.path.dirname(HERE), "include", "tpcca.h")]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-fmad=false", "-prec-div=true", "-prec-sqrt=true",
         "-Xcompiler", "-fPIC,-ffp-contract=off,-O2", "-Xptxas", "-v"]


def nvcc() -> str:
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def up_to_date(lib: str = LIB) -> bool:
    if not os.path.exists(lib):
        return False
    t = os.path.getmtime(lib)
    deps = [os.path.join(CSRC, s) for s in SOURCES] + HEADERS
    return all(os.path.getmtime(d) <= t for d in deps)


def build(force: bool = False, verbose: bool = False, checked: bool = False) -> str:
    lib, bdir = (LIB_CHECKED, BUILD_CHECKED) if checked else (LIB, BUILD)
    if not force and up_to_date(lib):
        return lib
    os.makedirs(bdir, exist_ok=True)
    cc = nvcc()
    procs = []
    extra = ["-DTPC_CHECKED"] if checked else []
    for src in SOURCES:
        obj = os.path.join(bdir, src.replace(".cu", ".o"))
        log = open(os.path.join(bdir, src + ".log"), "w")
        cmd = [cc, *ARCH, *FLAGS, *extra, "-c", os.path.join(CSRC, src), "-o", obj]
        procs.append((src, obj, log, subprocess.Popen(cmd, stdout=log, stderr=subprocess.STDOUT)))
    objs = []
    for src, obj, log, p in procs:
        rc = p.wait()
        log.close()
        text = open(log.name).read()
        if verbose:
            print(text)
        if rc != 0:
            raise RuntimeError("nvcc failed for %s:\n%s" % (src, text[-4000:]))
        objs.append(obj)
    tmp = lib + ".tmp%d" % os.getpid()
    subprocess.check_call([cc, *ARCH, "-shared", *objs, "-o", tmp, "-lcudart"])
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    print(build(force=True, verbose=True))
