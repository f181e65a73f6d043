"""The tensor-core operand store a SHT_MIXED plan uploads, checked on the host.

tc_build_images fills the store without zeroing it first, relying on the
packing to write every element.  tests/native/tc_images_check.cpp builds the
store into a buffer poisoned beforehand and compares it, op by op and in both
directions, with sht_plan_op_image; the op records' offsets must tile the
store exactly.  Compiled here with g++ against libsht.so (CPU only).
"""
import os
import shutil
import subprocess

import pytest

from paper_2004_11346_gb300 import _lib, build

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CUDA_INC = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "include")


@pytest.fixture(scope="module")
def checker(tmp_path_factory):
    if shutil.which("g++") is None or not os.path.exists(os.path.join(CUDA_INC, "cuda_runtime.h")):
        pytest.skip("g++ or the CUDA headers are missing")
    _lib.load()
    lib = build.LIB
    exe = str(tmp_path_factory.mktemp("tc") / "tc_images_check")
    cmd = ["g++", "-O1", "-std=c++17", "-I", os.path.join(ROOT, "paper_2004_11346_gb300", "csrc"),
           "-I", os.path.join(ROOT, "include"), "-I", CUDA_INC, os.path.join(HERE, "native", "tc_images_check.cpp"),
           "-o", exe, lib, "-Wl,-rpath," + os.path.dirname(lib)]
    subprocess.run(cmd, check=True, capture_output=True, text=True)
    return exe


@pytest.mark.parametrize("N,eps,n0,n_leaf,flags", [
    (40, 1e-7, 12, 6, _lib.SHT_FLAG_FORCE_FACTOR),   # butterflies: two-segment K sides
    (160, 1e-7, 80, 64, 0),                          # wide dense blocks: several 128-row tiles
    (96, 1e-7, 24, 16, 0),                           # default-like plan
])
def test_store_is_the_op_images(checker, N, eps, n0, n_leaf, flags):
    r = subprocess.run([checker, str(N), repr(eps), str(n0), str(n_leaf), str(flags)], capture_output=True,
                       text=True, timeout=600)
    assert r.returncode == 0, (r.returncode, r.stdout, r.stderr)
    assert r.stdout.startswith("ok ") and int(r.stdout.split()[1]) > 0
    # the live-row bound is checked on orders that have node rows no block
    # reaches (near the poles for large |m|), not only on full ones
    assert int(r.stdout.split()[2]) > 0
