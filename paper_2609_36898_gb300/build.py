"""Builds libvc.so in-tree: nvcc for sm_103a (CUDA sources) and the host encoder, linked into one
shared library next to this file. Translation units compile in parallel."""
from __future__ import annotations

import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libvc.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
# (source, object name, extra flags): the reconstruction kernels are compiled once per thread count
SOURCES = [("decode.cu", "decode", []), ("decode_nt.cu", "decode_nt256", ["-DVC_NT=256"]),
           ("decode_nt.cu", "decode_nt512", ["-DVC_NT=512"]), ("decode_nt.cu", "decode_nt1024", ["-DVC_NT=1024"]),
           ("vc_api.cu", "vc_api", []), ("decode_noalloc.cu", "decode_noalloc", []), ("encode.cpp", "encode", []),
           ("cache.cpp", "cache", []), ("server.cpp", "server", []),
           ("request.cu", "request", ["-Xcompiler", "-ffp-contract=off", "--fmad=false"]),
           ("render.cu", "render", ["-Xcompiler", "-ffp-contract=off", "--fmad=false"]),
           ("post.cu", "post", ["-Xcompiler", "-ffp-contract=off", "--fmad=false"]),
           ("frame.cu", "frame", ["-Xcompiler", "-ffp-contract=off", "--fmad=false"]),
           ("autotune.cpp", "autotune", []), ("split.cpp", "split", [])]
HEADERS = ["vc_internal.h", "decode_kernels.cuh", "cache.h"]


def _nvcc() -> str:
    for c in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc"):
        if c and os.path.exists(c):
            return c
    return "nvcc"


def _flags(src: str) -> list:
    common = ["-O3", "-std=c++17", "-I", INCLUDE, "-I", CSRC, "-Xcompiler", "-fPIC", "-Xcompiler", "-pthread"]
    if src.endswith(".cu"):
        return common + ARCH + ["-lineinfo", "-Xptxas", "-v"] if os.environ.get("VC_PTXAS_VERBOSE") else common + ARCH + ["-lineinfo"]
    return common + ["-x", "c++"]


def _stale(out: str, deps: list) -> bool:
    if not os.path.exists(out):
        return True
    t = os.path.getmtime(out)
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False) -> str:
    os.makedirs(BUILD, exist_ok=True)
    nvcc = _nvcc()
    hdrs = [os.path.join(CSRC, h) for h in HEADERS] + [os.path.join(INCLUDE, "vc.h")]
    jobs = []
    objs = []
    for s, name, extra in SOURCES:
        src = os.path.join(CSRC, s)
        obj = os.path.join(BUILD, name + ".o")
        objs.append(obj)
        if force or _stale(obj, [src] + hdrs + [__file__]):
            jobs.append([nvcc] + _flags(s) + extra + ["-c", src, "-o", obj])

    def run(cmd):
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("compile failed:\n" + " ".join(cmd) + "\n" + r.stdout + r.stderr)
        if verbose and (r.stdout or r.stderr):
            sys.stderr.write(r.stdout + r.stderr)

    with ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        list(ex.map(run, jobs))
    if force or jobs or _stale(LIB, objs):
        tmp = LIB + f".tmp{os.getpid()}"
        run([nvcc] + ARCH + ["-shared", "-o", tmp] + objs + ["-Xcompiler", "-pthread"])
        os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))
