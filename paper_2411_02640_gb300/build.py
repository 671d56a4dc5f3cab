"""In-tree build of libkx.so (the C-ABI library) for sm_103a.

Translation units are compiled in parallel; host-only sources go through
g++, the runtime through nvcc; the link uses nvcc so that the CUDA runtime
is linked statically and the library loads without a GPU present.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libkx.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def cuda_home() -> str:
    nvcc = shutil.which("nvcc")
    if nvcc:
        return os.path.dirname(os.path.dirname(os.path.realpath(nvcc)))
    return os.environ.get("CUDA_HOME", "/usr/local/cuda")


def _sources():
    return sorted(os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".cpp", ".cu")))


def _deps():
    return [os.path.join(CSRC, f) for f in os.listdir(CSRC)] + [os.path.join(ROOT, "include", "kx.h")]


def up_to_date() -> bool:
    if not os.path.exists(LIB):
        return False
    t = os.path.getmtime(LIB)
    return all(os.path.getmtime(d) <= t for d in _deps())


def build(force: bool = False, verbose: bool = False) -> str:
    if not force and up_to_date():
        return LIB
    os.makedirs(BUILD, exist_ok=True)
    ch = cuda_home()
    inc = ["-I", os.path.join(ROOT, "include"), "-I", CSRC, "-I", os.path.join(ch, "include")]
    jobs = []
    for src in _sources():
        obj = os.path.join(BUILD, os.path.basename(src) + ".o")
        if src.endswith(".cu"):
            cmd = ["nvcc", "-c", "-O2", "-std=c++17", "-Xcompiler", "-fPIC", "-lineinfo", *ARCH, *inc, src, "-o", obj]
        else:
            cmd = ["g++", "-c", "-O2", "-std=c++17", "-fPIC", "-Wall", *inc, src, "-o", obj]
        jobs.append((cmd, obj))

    def run(cmd):
        if verbose:
            print(" ".join(cmd), file=sys.stderr)
        subprocess.run(cmd, check=True)

    with cf.ThreadPoolExecutor(max_workers=max(1, len(jobs))) as ex:
        list(ex.map(run, [c for c, _ in jobs]))
    libdir = os.path.join(ch, "lib64")
    tmp = LIB + f".{os.getpid()}.tmp"
    run(["nvcc", "-shared", *ARCH, "-o", tmp, *[o for _, o in jobs], "-L", libdir, "-lnvrtc",
         "-Xlinker", "-rpath," + libdir])
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))
