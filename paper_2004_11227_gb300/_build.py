"""Build libcmf.so (the CUDA solver) in-tree with nvcc for sm_103a.

The translation units are compiled in parallel and linked into
``paper_2004_11227_gb300/libcmf.so``; objects go to ``paper_2004_11227_gb300/_build``.
The same batch builds ``libcmf_inject.so``, the fault-injection library of
the failure-detection tests: the translation units with bounded device waits
compiled again with CMF_FAULT_INJECTION (a short wait limit and a hook that
makes a wait run out), linked with the other objects.  Nothing on the product
path loads it.
"""
from __future__ import annotations

import glob
import os
import shutil
import subprocess

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
BUILD = os.path.join(PKG, "_build")
LIB = os.path.join(PKG, "libcmf.so")
LIB_INJECT = os.path.join(PKG, "libcmf_inject.so")
# translation units with bounded device waits (rebuilt for the injection library)
INJECT_TUS = ("cmf_binary_tma.cu", "cmf_potts_tma.cu")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr"]


def _nvcc() -> str:
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libcmf")


def sources() -> list:
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def _deps() -> list:
    return sources() + glob.glob(os.path.join(CSRC, "*.cuh")) + \
        [os.path.join(ROOT, "include", "cmf.h"), __file__]


def up_to_date() -> bool:
    if not os.path.exists(LIB) or not os.path.exists(LIB_INJECT):
        return False
    t = min(os.path.getmtime(LIB), os.path.getmtime(LIB_INJECT))
    return all(os.path.getmtime(d) <= t for d in _deps())


def build(force: bool = False, verbose: bool = False) -> str:
    """Compile every .cu under csrc/ and link libcmf.so; returns its path."""
    if not force and up_to_date():
        return LIB
    nvcc = _nvcc()
    os.makedirs(BUILD, exist_ok=True)
    procs = []
    objs = []
    inj_objs = []
    for src in sources():
        obj = os.path.join(BUILD, os.path.basename(src)[:-3] + ".o")
        objs.append(obj)
        cmd = [nvcc, *ARCH, *FLAGS, "-I", os.path.join(ROOT, "include"), "-c", src, "-o", obj]
        procs.append((src, subprocess.Popen(cmd, stdout=subprocess.PIPE,
                                            stderr=subprocess.STDOUT, text=True)))
        if os.path.basename(src) in INJECT_TUS:
            iobj = os.path.join(BUILD, os.path.basename(src)[:-3] + ".inject.o")
            inj_objs.append((obj, iobj))
            icmd = [nvcc, *ARCH, *FLAGS, "-DCMF_FAULT_INJECTION", "-I",
                    os.path.join(ROOT, "include"), "-c", src, "-o", iobj]
            procs.append((src + " (injection)",
                          subprocess.Popen(icmd, stdout=subprocess.PIPE,
                                           stderr=subprocess.STDOUT, text=True)))
    errors = []
    for src, p in procs:
        out, _ = p.communicate()
        if p.returncode != 0:
            errors.append(f"{os.path.basename(src)}:\n{out}")
        elif verbose and out:
            print(out)
    if errors:
        raise RuntimeError("nvcc failed:\n" + "\n".join(errors))
    tmp = LIB + ".tmp"
    subprocess.check_call([nvcc, *ARCH, "-shared", "-o", tmp, *objs])
    os.replace(tmp, LIB)
    swap = dict(inj_objs)
    tmp = LIB_INJECT + ".tmp"
    subprocess.check_call([nvcc, *ARCH, "-shared", "-o", tmp, *[swap.get(o, o) for o in objs]])
    os.replace(tmp, LIB_INJECT)
    return LIB


if __name__ == "__main__":
    print(build(force=True, verbose=True))
