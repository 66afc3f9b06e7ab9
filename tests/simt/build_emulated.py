"""Builds libhm_emu.so: the library with its CUDA kernels compiled as host
C++ (TEST INFRASTRUCTURE; see simt_prelude.h and simt_runtime.cpp).

The kernel sources are copied with two textual rewrites (applied to an
included kernel file too), since host
compilers know neither form: each ``kernel<<<grid, block, smem, stream>>>(args)``
becomes ``simt::launch(grid, block, smem, [&] { kernel(args); })``, and the
dynamic shared array ``extern __shared__ T name[];`` becomes a pointer to
the launch's buffer.  Nothing else in the sources changes.
"""
import os
import re
import shutil
import subprocess
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
CSRC = os.path.join(ROOT, "paper_1910_09142_gb300", "csrc")
KERNELS = ("hm_fp64.cu", "hm_mixed.cu", "hm_mixed_pair.cu")
# test-only kernel sources (this folder), rewritten the same way
PROBES = ("block_harness.cu",)


def rewrite(text):
    # a kernel file that builds another one with different settings
    # (#define ..., #include "other.cu") gets that file's rewritten text
    def include(m):
        with open(os.path.join(CSRC, m.group(1))) as f:
            return rewrite(f.read())
    text = re.sub(r'#include "(\w+\.cu)"', include, text)

    def launch(m):
        config = ",".join(m.group(2).split(",")[:3])          # grid, block, smem (stream dropped)
        return "simt::launch(%s, [&] { %s(%s); });" % (config, m.group(1), m.group(3))
    text = re.sub(r"(\w+)<<<([^>]*?)>>>\((.*?)\);", launch, text, flags=re.S)
    return re.sub(r"extern __shared__ (\w+) (\w+)\[\];", r"\1* \2 = (\1*)simt::dynamic_smem();", text)


def build(out_dir, cxx=None):
    """Compile into out_dir; returns the library path.  Raises on failure."""
    cxx = cxx or shutil.which("g++")
    inc = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "include")
    if not cxx or not os.path.exists(os.path.join(inc, "cuda_runtime.h")):
        raise FileNotFoundError("needs g++ and the CUDA headers")
    flags = ["-std=c++20", "-O2", "-fPIC", "-I" + inc, "-I" + CSRC]
    objs = []
    jobs = []
    for name in KERNELS + PROBES:
        src = os.path.join(out_dir, name.replace(".cu", ".cpp"))
        with open(os.path.join(CSRC if name in KERNELS else HERE, name)) as f:
            text = rewrite(f.read())
        with open(src, "w") as f:
            f.write(text)
        obj = src.replace(".cpp", ".o")
        objs.append(obj)
        jobs.append([cxx, *flags, "-include", os.path.join(HERE, "simt_prelude.h"), "-c", src, "-o", obj])
    host = [os.path.join(CSRC, "hm_api.cu"), os.path.join(HERE, "simt_runtime.cpp"),
            os.path.join(ROOT, "tests", "host_abi", "cuda_runtime_stub.cpp")]
    for src in host:
        obj = os.path.join(out_dir, os.path.basename(src) + ".o")
        objs.append(obj)
        jobs.append([cxx, *flags, "-x", "c++", "-c", src, "-o", obj])
    with ThreadPoolExecutor(len(jobs)) as pool:
        results = list(pool.map(lambda cmd: subprocess.run(cmd, capture_output=True, text=True), jobs))
    for cmd, r in zip(jobs, results):
        if r.returncode:
            raise RuntimeError("%s failed:\n%s" % (os.path.basename(cmd[-3]), r.stderr[-4000:]))
    lib = os.path.join(out_dir, "libhm_emu.so")
    r = subprocess.run([cxx, "-shared", "-o", lib, *objs, "-ldl", "-Wl,-Bsymbolic"], capture_output=True, text=True)
    if r.returncode:
        raise RuntimeError("link failed:\n" + r.stderr[-4000:])
    return lib
