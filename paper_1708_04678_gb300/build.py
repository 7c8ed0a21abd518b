"""Build ``libfelbm.so`` (the C-ABI CUDA library) in-tree with nvcc for sm_103a.

    python -m paper_1708_04678_gb300.build

The library is rebuilt when a source or header changed since the last build
(a stamp file holds the hash of the sources, the flags and the machine).
"""
from __future__ import annotations

import hashlib
import os
import platform
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
LIBDIR = os.path.join(PKG, "lib")
LIBNAME = "libfelbm.so"
SOURCES = ["mesh.cpp", "felbm.cu", "mesh3d.cpp", "felbm3d.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-Xcompiler", "-O3"]


def nvcc_path():
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libfelbm.so")


def lib_path():
    return os.path.join(LIBDIR, LIBNAME)


def _stamp():
    h = hashlib.sha256()
    for d in (CSRC, INCLUDE):
        for name in sorted(os.listdir(d)):
            if name.endswith((".cu", ".cpp", ".h", ".cuh")):
                with open(os.path.join(d, name), "rb") as f:
                    h.update(name.encode())
                    h.update(f.read())
    h.update(" ".join(ARCH + FLAGS).encode())
    h.update(platform.machine().encode())
    return h.hexdigest()


def build(force=False, verbose=False):
    """Compile every translation unit in parallel and link the shared library."""
    os.makedirs(LIBDIR, exist_ok=True)
    stamp_file = os.path.join(LIBDIR, "build.stamp")
    stamp = _stamp()
    if not force and os.path.exists(lib_path()) and os.path.exists(stamp_file):
        with open(stamp_file) as f:
            if f.read().strip() == stamp:
                return lib_path()
    nvcc = nvcc_path()
    objs = []
    cmds = []
    for name in SOURCES:
        obj = os.path.join(LIBDIR, name + ".o")
        objs.append(obj)
        cmds.append([nvcc, *ARCH, *FLAGS, "-I", INCLUDE, "-I", CSRC, "-c",
                     os.path.join(CSRC, name), "-o", obj])

    def run(cmd):
        if verbose:
            print(" ".join(cmd), flush=True)
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("nvcc failed:\n" + " ".join(cmd) + "\n" + r.stdout + r.stderr)
        return r.stdout + r.stderr

    with ThreadPoolExecutor(max_workers=len(cmds)) as ex:
        logs = list(ex.map(run, cmds))
    if verbose:
        for lg in logs:
            if lg.strip():
                print(lg)
    tmp = lib_path() + ".tmp"
    run([nvcc, *ARCH, "-shared", "-o", tmp, *objs])
    os.replace(tmp, lib_path())
    with open(stamp_file, "w") as f:
        f.write(stamp)
    return lib_path()


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))
