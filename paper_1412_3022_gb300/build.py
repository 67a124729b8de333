"""Builds libpmrc.so in-tree with nvcc for sm_103a (GB300).

The CUDA translation units and the host C++ sources are compiled in
parallel, then linked into one shared library next to this file.  No
PyTorch extension machinery is involved: the library exposes a plain C ABI
(include/pmrc.h) and the Python binding loads it with ctypes.
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
OUT = os.path.join(HERE, "libpmrc.so")
BUILD = os.path.join(ROOT, "_build")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
SOURCES = ["bitslice_k16.cu", "bitslice_k12.cu", "region.cu", "bitslice.cu", "repair.cu", "batch.cu", "serve.cu", "plan.cpp",
           "code.cpp", "code16.cpp", "specific.cpp", "bs_emit.cpp", "jit.cpp", "api.cpp"]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libpmrc")


def _stale() -> bool:
    if not os.path.exists(OUT):
        return True
    t = os.path.getmtime(OUT)
    for d in (CSRC, os.path.join(ROOT, "include")):
        for f in os.listdir(d):
            if os.path.getmtime(os.path.join(d, f)) > t:
                return True
    return os.path.getmtime(__file__) > t


def build(force: bool = False, verbose: bool = False) -> str:
    if not force and not _stale():
        return OUT
    os.makedirs(BUILD, exist_ok=True)
    cc = nvcc()
    # 1. generate the bitsliced encode schedules with the library's own
    #    host construction (gen_bitslice.cpp + code.cpp, plain g++)
    gen = os.path.join(BUILD, "gen_bitslice")
    cxx = shutil.which("g++") or "g++"
    r = subprocess.run([cxx, "-std=c++17", "-O2", "-I" + CSRC, "-o", gen,
                        os.path.join(CSRC, "gen_bitslice.cpp"), os.path.join(CSRC, "bs_emit.cpp"),
                        os.path.join(CSRC, "code.cpp"), os.path.join(CSRC, "code16.cpp")],
                       capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"g++ failed on gen_bitslice:\n{r.stdout}\n{r.stderr}")
    r = subprocess.run([gen, os.path.join(BUILD, "bitslice_gen.cuh"),
                        os.path.join(BUILD, "bitslice_gen_k12.cuh"),
                        os.path.join(BUILD, "bitslice_gen_k16.cuh")], capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"gen_bitslice failed:\n{r.stdout}\n{r.stderr}")
    # 2. the bitsliced device code as a string, for run-time compilation
    with open(os.path.join(CSRC, "bitslice_dev.cuh")) as f:
        dev_src = f.read()
    if ")BSDEV\"" in dev_src:
        raise RuntimeError("bitslice_dev.cuh contains the raw-string delimiter")
    with open(os.path.join(BUILD, "bitslice_dev_src.inc"), "w") as f:
        f.write('static const char kBsDevSrc[] = R"BSDEV(' + dev_src + ')BSDEV";\n')
    common = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC,-O2",
                     "-I" + os.path.join(ROOT, "include"), "-I" + CSRC, "-I" + BUILD]

    def compile_one(src: str) -> str:
        obj = os.path.join(BUILD, src + ".o")
        cmd = [cc] + common + ["-c", os.path.join(CSRC, src), "-o", obj]
        if src.endswith(".cu"):
            cmd += ["-Xptxas", "-v"] if verbose else []
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {src}:\n{r.stdout}\n{r.stderr}")
        if verbose and r.stderr:
            sys.stderr.write(r.stderr)
        return obj

    with cf.ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        objs = list(ex.map(compile_one, SOURCES))
    tmp = OUT + f".tmp{os.getpid()}"
    cmd = [cc] + ARCH + ["-shared", "-o", tmp] + objs + ["-lpthread", "-ldl"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, OUT)
    return OUT


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
