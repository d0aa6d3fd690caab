"""Builds libcbvh.so in-tree: host builder (g++) and sm_103a kernels (nvcc), compiled in
parallel and linked into one shared library with a static CUDA runtime."""
from __future__ import annotations

import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
LIB = os.path.join(HERE, "libcbvh.so")
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
    if not os.path.exists(LIB):
        return False
    t = os.path.getmtime(LIB)
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
    cmds = (host_cmd, dev_cmd, refit_cmd, devbuild_cmd, probe_cmd)
    procs = [subprocess.Popen(c, stdout=subprocess.PIPE, stderr=subprocess.STDOUT, text=True) for c in cmds]
    outs = [p.communicate()[0] for p in procs]
    for p, c, o in zip(procs, cmds, outs):
        if p.returncode != 0:
            raise RuntimeError(f"build failed: {' '.join(c)}\n{o}")
        if verbose and o:
            print(o)
    tmp = LIB + f".tmp{os.getpid()}"
    link = [nvcc, *ARCH, "-shared", "-cudart", "static", "-o", tmp, obj_host, obj_dev, obj_refit, obj_devbuild,
            obj_probe]
    r = subprocess.run(link, stdout=subprocess.PIPE, stderr=subprocess.STDOUT, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed: {' '.join(link)}\n{r.stdout}")
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    import sys
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
