"""Builds the in-tree shared library ``_build/libfse.so`` for sm_103a.

nvcc compiles the kernels and g++ the host sources in parallel, then nvcc
links the shared library against the CUDA runtime.  No CMake, one -gencode.
"""
import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(OUT_DIR, "libfse.so")
ROOT = os.path.dirname(HERE)

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
CU_SRC = ["fse_kernels.cu", "fse_noalloc.cu"]
CPP_SRC = ["fse_api.cpp", "fse_abi.cpp", "fse_server.cpp"]


def _cuda_home():
    for c in (os.environ.get("CUDA_HOME"), "/usr/local/cuda"):
        if c and os.path.exists(os.path.join(c, "bin", "nvcc")):
            return c
    nv = shutil.which("nvcc")
    if nv:
        return os.path.dirname(os.path.dirname(nv))
    raise RuntimeError("nvcc not found")


def _run(cmd):
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("build step failed:\n" + " ".join(cmd) + "\n" + r.stdout + r.stderr)
    return r.stdout + r.stderr


def build(force=False, verbose=False):
    srcs = [os.path.join(CSRC, s) for s in CU_SRC + CPP_SRC]
    hdrs = [os.path.join(CSRC, h) for h in os.listdir(CSRC) if h.endswith(".h")]
    hdrs.append(os.path.join(ROOT, "include", "fse.h"))
    if not force and os.path.exists(LIB):
        t = os.path.getmtime(LIB)
        if all(os.path.getmtime(s) <= t for s in srcs + hdrs):
            return LIB
    os.makedirs(OUT_DIR, exist_ok=True)
    cuda = _cuda_home()
    nvcc = os.path.join(cuda, "bin", "nvcc")
    inc = ["-I", os.path.join(cuda, "include"), "-I", CSRC, "-I", os.path.join(ROOT, "include")]
    jobs = []
    for s in CU_SRC:
        o = os.path.join(OUT_DIR, s + ".o")
        jobs.append(([nvcc] + ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC",
                                       "-Xptxas", "-v", "-c", os.path.join(CSRC, s), "-o", o] + inc, o))
    for s in CPP_SRC:
        o = os.path.join(OUT_DIR, s + ".o")
        jobs.append((["g++", "-O2", "-std=c++17", "-fPIC", "-Wall", "-c", os.path.join(CSRC, s),
                      "-o", o] + inc, o))
    with cf.ThreadPoolExecutor(max_workers=len(jobs)) as ex:
        logs = list(ex.map(lambda j: _run(j[0]), jobs))
    if verbose:
        for l in logs:
            sys.stdout.write(l)
    tmp = LIB + ".tmp"
    _run([nvcc] + ARCH + ["-shared", "-o", tmp] + [o for _, o in jobs] +
         ["-lcudart", "-lpthread"])
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
