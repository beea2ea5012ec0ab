"""Build libgadep.so in-tree: host C++ with g++, CUDA with nvcc for sm_103a only.

    python -m paper_2605_25963_gb300.build [--force]

Translation units compile in parallel; the result is
``paper_2605_25963_gb300/lib/libgadep.so`` (git-ignored).
"""
from __future__ import annotations

import concurrent.futures as cf
import hashlib
import os
import shutil
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
OUT_DIR = os.path.join(PKG, "lib")
LIB = os.path.join(OUT_DIR, "libgadep.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]

CXX_SOURCES = ["detmesh.cpp", "geometry.cpp", "xs.cpp", "bvh.cpp"]
CU_SOURCES = ["transport.cu", "wavefront.cu"]


def _cuda_home() -> str:
    for c in (os.environ.get("CUDA_HOME"), "/usr/local/cuda"):
        if c and os.path.exists(os.path.join(c, "bin", "nvcc")):
            return c
    nvcc = shutil.which("nvcc")
    if nvcc:
        return os.path.dirname(os.path.dirname(nvcc))
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libgadep")


def _inputs_digest() -> str:
    h = hashlib.sha256()
    for d, names in ((CSRC, sorted(os.listdir(CSRC))), (INCLUDE, sorted(os.listdir(INCLUDE)))):
        for n in names:
            p = os.path.join(d, n)
            if os.path.isfile(p):
                h.update(n.encode())
                with open(p, "rb") as f:
                    h.update(f.read())
    h.update(open(__file__, "rb").read())
    return h.hexdigest()


def build(force: bool = False, verbose: bool = False) -> str:
    digest = _inputs_digest()
    stamp = os.path.join(OUT_DIR, "build.stamp")
    if not force and os.path.exists(LIB) and os.path.exists(stamp):
        if open(stamp).read().strip() == digest:
            return LIB
    os.makedirs(OUT_DIR, exist_ok=True)
    cuda = _cuda_home()
    nvcc = os.path.join(cuda, "bin", "nvcc")
    inc = ["-I", INCLUDE, "-I", CSRC, "-I", os.path.join(cuda, "include")]
    jobs = []
    objs = []
    for s in CXX_SOURCES:
        o = os.path.join(OUT_DIR, s + ".o")
        objs.append(o)
        jobs.append(["g++", "-std=c++17", "-O2", "-fPIC", "-Wall", "-Wno-unused-function", "-c",
                     os.path.join(CSRC, s), "-o", o] + inc)
    for s in CU_SOURCES:
        o = os.path.join(OUT_DIR, s + ".o")
        objs.append(o)
        jobs.append([nvcc, "-std=c++17", "-O3", "-lineinfo", "-Xcompiler", "-fPIC",
                     "--expt-relaxed-constexpr", "-Xptxas", "-v"] + ARCH + ["-c", os.path.join(CSRC, s),
                                                                           "-o", o] + inc)

    def run(cmd):
        r = subprocess.run(cmd, capture_output=True, text=True)
        return cmd, r

    logs = []
    with cf.ThreadPoolExecutor(max_workers=max(1, min(len(jobs), os.cpu_count() or 1))) as ex:
        for cmd, r in ex.map(run, jobs):
            if r.returncode != 0:
                raise RuntimeError("compile failed: %s\n%s\n%s" % (" ".join(cmd), r.stdout, r.stderr))
            if verbose and (r.stdout or r.stderr):
                print(r.stdout + r.stderr, file=sys.stderr)
            if "-Xptxas" in cmd:
                logs.append(r.stdout + r.stderr)
    with open(os.path.join(OUT_DIR, "ptxas.log"), "w") as f:
        f.write("\n".join(logs))
    tmp = LIB + ".tmp.%d" % os.getpid()
    link = [nvcc, "-shared"] + ARCH + objs + ["-o", tmp, "-lcudart_static", "-lpthread", "-ldl", "-lrt"]
    r = subprocess.run(link, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("link failed: %s\n%s" % (r.stdout, r.stderr))
    os.replace(tmp, LIB)
    with open(stamp, "w") as f:
        f.write(digest)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))
