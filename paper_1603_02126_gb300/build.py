"""Build libepic.so in-tree for sm_103a (nvcc + g++, no cmake).

    python -m paper_1603_02126_gb300.build        # or __graft_entry__.build()

Objects and the library go to paper_1603_02126_gb300/_lib/ (git-ignored).
Translation units compile in parallel; a rebuild happens only when a source
or header is newer than the library.
"""
from __future__ import annotations

import os
import shutil
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
OUT = os.path.join(PKG, "_lib")
LIB = os.path.join(OUT, "libepic.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]

CU_SOURCES = ["epic_kernels.cu", "epic_unfused.cu", "epic_tc.cu", "epic_cluster.cu", "epic_noalloc.cu",
              "epic_piped.cu", "epic_peak.cu", "epic_multipix.cu", "epic_xengine.cu", "epic_adjoint.cu"]
CXX_SOURCES = ["epic_plan.cpp"]
HEADERS = [os.path.join(CSRC, "epic_internal.h"), os.path.join(CSRC, "epic_fft.cuh"),
           os.path.join(CSRC, "epic_fused_geo.cuh"),
           os.path.join(ROOT, "include", "epic.h")]


def _cuda_home() -> str:
    for cand in (os.environ.get("CUDA_HOME"), "/usr/local/cuda"):
        if cand and os.path.exists(os.path.join(cand, "bin", "nvcc")):
            return cand
    nvcc = shutil.which("nvcc")
    if nvcc:
        return os.path.dirname(os.path.dirname(nvcc))
    raise RuntimeError("nvcc not found: set CUDA_HOME")


def _stale(target: str, deps) -> bool:
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps)


def build(verbose: bool = False, force: bool = False) -> str:
    """Compile every translation unit for sm_103a and link libepic.so."""
    cuda = _cuda_home()
    nvcc = os.path.join(cuda, "bin", "nvcc")
    os.makedirs(OUT, exist_ok=True)
    srcs = [os.path.join(CSRC, s) for s in CU_SOURCES + CXX_SOURCES]
    if not force and not _stale(LIB, srcs + HEADERS + [os.path.abspath(__file__)]):
        return LIB
    inc = ["-I" + os.path.join(ROOT, "include"), "-I" + CSRC, "-I" + os.path.join(cuda, "include")]
    jobs = []
    objs = []
    for s in CU_SOURCES:
        o = os.path.join(OUT, s + ".o")
        objs.append(o)
        cmd = [nvcc, *ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC",
               "-Xcompiler", "-ffp-contract=off", *inc, "-c", os.path.join(CSRC, s), "-o", o]
        jobs.append(cmd)
    for s in CXX_SOURCES:
        o = os.path.join(OUT, s + ".o")
        objs.append(o)
        cmd = ["g++", "-O2", "-std=c++17", "-fPIC", "-ffp-contract=off", "-Wall", *inc, "-c",
               os.path.join(CSRC, s), "-o", o]
        jobs.append(cmd)
    procs = [(cmd, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT, text=True))
             for cmd in jobs]
    failed = []
    for cmd, pr in procs:
        out, _ = pr.communicate()
        if verbose and out:
            print(out)
        if pr.returncode != 0:
            failed.append((cmd, out))
    if failed:
        msg = "\n".join(" ".join(c) + "\n" + o for c, o in failed)
        raise RuntimeError("libepic build failed:\n" + msg)
    tmp = LIB + ".tmp"
    link = [nvcc, *ARCH, "-shared", "-cudart", "static", "-o", tmp, *objs, "-ldl"]
    r = subprocess.run(link, stdout=subprocess.PIPE, stderr=subprocess.STDOUT, text=True)
    if r.returncode != 0:
        raise RuntimeError("libepic link failed:\n" + " ".join(link) + "\n" + r.stdout)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(verbose="-v" in sys.argv, force="-f" in sys.argv))
