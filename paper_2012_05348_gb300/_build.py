"""Builds libcbvh.so in-tree: host builder (g++) and sm_103a kernels (nvcc), compiled in
parallel and linked into one shared library with a static CUDA runtime.  Beside it,
libcbvh_checked.so: the same library with the traversal compiled with CBVH_CHECKED (every
index read from a blob or computed by the traversal bounds-checked into the status word),
loaded instead when the environment sets CBVH_CHECKED=1."""
from __future__ import annotations

import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
LIB = os.path.join(HERE, "libcbvh.so")
LIB_CHECKED = os.path.join(HERE, "libcbvh_checked.so")
BUILD_DIR = os.path.join(HERE, "_build")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def _nvcc() -> str:
    cand = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(cand):
        raise RuntimeError("nvcc not found (CUDA toolkit required to build libcbvh)")
    return cand


def sources():
    return [os.path.join(CSRC, f) for f in ("build.cpp", "kernels.cu", "refit.cu", "devbuild.cu", "probe.cu", "internal.h",
                                            "lattice.cuh")] + [
        os.path.join(INCLUDE, "cbvh.h")]


def up_to_date() -> bool:
    if not os.path.exists(LIB) or not os.path.exists(LIB_CHECKED):
        return False
    t = min(os.path.getmtime(LIB), os.path.getmtime(LIB_CHECKED))
    return all(os.path.getmtime(s) <= t for s in sources())


def build(force: bool = False, verbose: bool = False) -> str:
    if not force and up_to_date():
        return LIB
    os.makedirs(BUILD_DIR, exist_ok=True)
    nvcc = _nvcc()
    obj_host = os.path.join(BUILD_DIR, "build.o")
    obj_dev = os.path.join(BUILD_DIR, "kernels.o")
    obj_refit = os.path.join(BUILD_DIR, "refit.o")
    obj_devbuild = os.path.join(BUILD_DIR, "devbuild.o")
    obj_probe = os.path.join(BUILD_DIR, "probe.o")
    host_cmd = ["g++", "-O2", "-std=c++17", "-fPIC", "-ffp-contract=off", "-Wall", "-I", INCLUDE, "-c",
                os.path.join(CSRC, "build.cpp"), "-o", obj_host]
    dev_cmd = [nvcc, "-O3", "-std=c++17", *ARCH, "-lineinfo", "-Xcompiler", "-fPIC,-ffp-contract=off",
               "-Xptxas", "-v" if verbose else "-O3", "-I", INCLUDE, "-c", os.path.join(CSRC, "kernels.cu"),
               "-o", obj_dev]
    refit_cmd = dev_cmd[:-4] + ["-c", os.path.join(CSRC, "refit.cu"), "-o", obj_refit]
    devbuild_cmd = dev_cmd[:-4] + ["-c", os.path.join(CSRC, "devbuild.cu"), "-o", obj_devbuild]
    probe_cmd = dev_cmd[:-4] + ["-c", os.path.join(CSRC, "probe.cu"), "-o", obj_probe]
    obj_checked = os.path.join(BUILD_DIR, "kernels_checked.o")
    checked_cmd = dev_cmd[:-4] + ["-DCBVH_CHECKED", "-c", os.path.join(CSRC, "kernels.cu"), "-o", obj_checked]
    cmds = (host_cmd, dev_cmd, refit_cmd, devbuild_cmd, probe_cmd, checked_cmd)
    procs = [subprocess.Popen(c, stdout=subprocess.PIPE, stderr=subprocess.STDOUT, text=True) for c in cmds]
    outs = [p.communicate()[0] for p in procs]
    for p, c, o in zip(procs, cmds, outs):
        if p.returncode != 0:
            raise RuntimeError(f"build failed: {' '.join(c)}\n{o}")
        if verbose and o:
            print(o)
    for lib, kobj in ((LIB_CHECKED, obj_checked), (LIB, obj_dev)):
        tmp = lib + f".tmp{os.getpid()}"
        link = [nvcc, *ARCH, "-shared", "-cudart", "static", "-o", tmp, obj_host, kobj, obj_refit, obj_devbuild,
                obj_probe]
        r = subprocess.run(link, stdout=subprocess.PIPE, stderr=subprocess.STDOUT, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"link failed: {' '.join(link)}\n{r.stdout}")
        os.replace(tmp, lib)
    return LIB


if __name__ == "__main__":
    import sys
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
