"""Build libmbs.so in-tree: CUDA kernels for sm_103a (nvcc) plus the host
setup and C ABI (g++ with OpenMP), compiled in parallel and linked against
the shared CUDA runtime."""
from __future__ import annotations

import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "_build")
LIB = os.path.join(OUT, "libmbs.so")
ROOT = os.path.dirname(HERE)
CUDA = os.environ.get("CUDA_HOME", "/usr/local/cuda")
NVCC = os.path.join(CUDA, "bin", "nvcc")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]

SOURCES_CU = ["mbs_tiled.cu", "mbs_tc.cu", "mbs_cells.cu", "mbs_plain.cu", "mbs_plain45.cu", "mbs_plain6.cu",
              "mbs_static.cu", "mbs_peaks.cu", "mbs_setup_dev.cu"]
SOURCES_CPP = ["mbs_setup.cpp", "mbs_host.cpp", "mbs_solve.cpp", "mbs_batch.cpp", "mbs_cells_host.cpp"]
HEADERS = ["mbs_internal.h", "mbs_device.cuh", "mbs_host_internal.h", "mbs_step_math.h", "mbs_setup_dev.h"]


def _stale(target, deps):
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False, extra_nvcc=()) -> str:
    os.makedirs(OUT, exist_ok=True)
    hdrs = [os.path.join(CSRC, h) for h in HEADERS] + [os.path.join(ROOT, "include", "mbs.h")]
    jobs, objs = [], []
    for s in SOURCES_CU:
        src = os.path.join(CSRC, s)
        obj = os.path.join(OUT, s + ".o")
        objs.append(obj)
        if force or _stale(obj, [src] + hdrs):
            cmd = [NVCC, *ARCH, "-lineinfo", "-O3", "-std=c++17", "-Xcompiler", "-fPIC",
                   "-Xptxas", "-v" if verbose else "-O3", *extra_nvcc, "-c", src, "-o", obj]
            jobs.append((cmd, s))
    for s in SOURCES_CPP:
        src = os.path.join(CSRC, s)
        obj = os.path.join(OUT, s + ".o")
        objs.append(obj)
        if force or _stale(obj, [src] + hdrs):
            cmd = ["g++", "-O2", "-std=c++17", "-fPIC", "-fopenmp", "-I" + os.path.join(CUDA, "include"),
                   "-c", src, "-o", obj]
            jobs.append((cmd, s))
    procs = [(subprocess.Popen(c, stdout=subprocess.PIPE, stderr=subprocess.STDOUT, text=True), s)
             for c, s in jobs]
    failed = []
    for p, s in procs:
        out, _ = p.communicate()
        if verbose or p.returncode:
            sys.stderr.write(out)
        if p.returncode:
            failed.append(s)
    if failed:
        raise RuntimeError(f"compilation failed: {failed}")
    if force or jobs or not os.path.exists(LIB):
        tmp = LIB + f".{os.getpid()}.tmp"
        subprocess.check_call([NVCC, *ARCH, "-shared", "-cudart", "shared", "-o", tmp, *objs,
                               "-Xcompiler", "-fopenmp", "-lgomp",
                               "-Xlinker", "-rpath=" + os.path.join(CUDA, "lib64")])
        os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
