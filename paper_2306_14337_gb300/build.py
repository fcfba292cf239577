"""Build the CUDA library ``libkkt.so`` in-tree for sm_103a (GB300).

Two translation units compile in parallel: the host analysis with g++ and the
kernels plus C entry points with nvcc; nvcc links them into a shared library
with the CUDA runtime linked statically.
"""
from __future__ import annotations

import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(OUT_DIR, "libkkt.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def _nvcc():
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def sources():
    return [os.path.join(CSRC, f) for f in ("analysis.cpp", "kkt.cu", "dense.cu", "noalloc.cu", "probe.cu")] + [
        os.path.join(CSRC, f) for f in ("analysis.h", "kernels.cuh")] + [os.path.join(INCLUDE, "kkt.h")]


def up_to_date():
    if not os.path.exists(LIB):
        return False
    t = os.path.getmtime(LIB)
    return all(os.path.getmtime(s) <= t for s in sources())


def build(force: bool = False, verbose: bool = False) -> str:
    if not force and up_to_date():
        return LIB
    os.makedirs(OUT_DIR, exist_ok=True)
    nvcc = _nvcc()
    tag = str(os.getpid())
    o_host = os.path.join(OUT_DIR, f"analysis.{tag}.o")
    o_dev = os.path.join(OUT_DIR, f"kkt.{tag}.o")
    o_na = os.path.join(OUT_DIR, f"noalloc.{tag}.o")
    o_pr = os.path.join(OUT_DIR, f"probe.{tag}.o")
    o_dn = os.path.join(OUT_DIR, f"dense.{tag}.o")
    cuda = [nvcc, "-O3", "-std=c++17", *ARCH, "-lineinfo", "-Xcompiler", "-fPIC", "-I", INCLUDE, "-c"]
    cmds = [
        ["g++", "-O2", "-std=c++17", "-fPIC", "-I", INCLUDE, "-c", os.path.join(CSRC, "analysis.cpp"),
         "-o", o_host],
        cuda + [os.path.join(CSRC, "kkt.cu"), "-o", o_dev],
        cuda + [os.path.join(CSRC, "noalloc.cu"), "-o", o_na],
        cuda + [os.path.join(CSRC, "probe.cu"), "-o", o_pr],
        cuda + [os.path.join(CSRC, "dense.cu"), "-o", o_dn],
    ]
    procs = [subprocess.Popen(c, stdout=subprocess.PIPE, stderr=subprocess.STDOUT, text=True) for c in cmds]
    outs = [p.communicate()[0] for p in procs]
    for c, p, o in zip(cmds, procs, outs):
        if verbose or p.returncode:
            sys.stderr.write(" ".join(c) + "\n" + o)
        if p.returncode:
            raise RuntimeError(f"compile failed: {c[0]} ({p.returncode})")
    tmp = LIB + f".{tag}.tmp"
    link = [nvcc, "-shared", *ARCH, "-o", tmp, o_host, o_dev, o_na, o_pr, o_dn, "-lpthread", "-ldl"]
    r = subprocess.run(link, stdout=subprocess.PIPE, stderr=subprocess.STDOUT, text=True)
    if verbose or r.returncode:
        sys.stderr.write(" ".join(link) + "\n" + r.stdout)
    if r.returncode:
        raise RuntimeError("link failed")
    os.replace(tmp, LIB)
    for o in (o_host, o_dev, o_na, o_pr, o_dn):
        os.remove(o)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))
