"""Build libsht.so in-tree for sm_103a (GB300).

Two translation units compiled in parallel: the host plan builder (g++,
OpenMP) and the CUDA kernels with the C ABI (nvcc, sm_103a), linked into
``paper_2004_11346_gb300/_build/libsht.so``.
"""
from __future__ import annotations

import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "libsht.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]

HOST_SRC = ["plan.cpp"]
CUDA_SRC = ["apply.cu", "apply_f32.cu", "apply_tc.cu", "phi_dft.cu", "alt_direct.cu"]


def cuda_home() -> str:
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    return os.path.dirname(os.path.dirname(os.path.realpath(nvcc)))


def _sources():
    out = [os.path.join(CSRC, f) for f in os.listdir(CSRC)]
    out += [os.path.join(INCLUDE, f) for f in os.listdir(INCLUDE)]
    return out + [os.path.abspath(__file__)]


def stale() -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    return any(os.path.getmtime(s) > t for s in _sources())


def build(force: bool = False, verbose: bool = False) -> str:
    if not force and not stale():
        return LIB
    os.makedirs(BUILD, exist_ok=True)
    home = cuda_home()
    nvcc = os.path.join(home, "bin", "nvcc")
    if not os.path.exists(nvcc):
        nvcc = "nvcc"
    inc = ["-I", CSRC, "-I", INCLUDE]
    jobs = []
    objs = []
    for f in HOST_SRC:
        o = os.path.join(BUILD, f + ".o")
        objs.append(o)
        jobs.append(["g++", "-O3", "-std=c++17", "-fopenmp", "-fPIC", "-Wall", "-Wno-unused-function",
                     *inc, "-c", os.path.join(CSRC, f), "-o", o])
    for f in CUDA_SRC:
        o = os.path.join(BUILD, f + ".o")
        objs.append(o)
        jobs.append([nvcc, *ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC",
                     "--expt-relaxed-constexpr", "-Xcompiler", "-fopenmp", *inc, "-c", os.path.join(CSRC, f), "-o", o])
    procs = [subprocess.Popen(j, stdout=subprocess.PIPE, stderr=subprocess.STDOUT) for j in jobs]
    errors = []
    for j, p in zip(jobs, procs):
        out, _ = p.communicate()
        if p.returncode != 0 or verbose:
            (errors if p.returncode != 0 else []).append(" ".join(j) + "\n" + out.decode())
            if verbose:
                print(out.decode())
    if errors:
        raise RuntimeError("libsht build failed:\n" + "\n".join(errors))
    libdirs = [os.path.join(home, "lib64"), os.path.join(home, "lib")]
    libdirs += [os.path.join(home, "targets", t, "lib") for t in ("sbsa-linux", "x86_64-linux", "aarch64-linux")]
    libdirs = [d for d in libdirs if os.path.isdir(d)]
    tmp = LIB + f".tmp{os.getpid()}"
    link = ["g++", "-shared", "-fopenmp", "-o", tmp, *objs]
    for d in libdirs:
        link += ["-L", d, f"-Wl,-rpath,{d}"]
    link += ["-lcudart"]
    subprocess.run(link, check=True)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force=True, verbose=True))
