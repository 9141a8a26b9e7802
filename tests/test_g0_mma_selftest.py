"""One tcgen05 MMA in isolation: shared-memory descriptors, instruction
descriptor and TMEM read-back conventions that every tensor-core kernel
relies on.  Runs before the evaluation tests.  The kernel lives in a
test-only library (tests/native/mma_selftest.cu), built here with nvcc."""
import ctypes as C
import os
import subprocess

import numpy as np
import pytest

from conftest import kmajor_pack

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "native", "mma_selftest.cu")
LIB = os.path.join(HERE, "native", "_build", "libmma_selftest.so")


@pytest.fixture(scope="module")
def lib():
    if not os.path.exists(LIB) or os.path.getmtime(LIB) < os.path.getmtime(SRC):
        os.makedirs(os.path.dirname(LIB), exist_ok=True)
        subprocess.check_call(["/usr/local/cuda/bin/nvcc", "-gencode", "arch=compute_103a,code=sm_103a", "-O2",
                               "-std=c++17", "-Xcompiler", "-fPIC", "-shared", "-o", LIB, SRC])
    L = C.CDLL(LIB)
    L.mma_selftest.restype = C.c_int
    L.mma_selftest.argtypes = [C.c_void_p] * 3 + [C.c_int]
    return L


def _run(lib, A_bits, B_bits, a_in_tmem):
    A = np.ascontiguousarray(A_bits, dtype=np.uint16)
    B = np.ascontiguousarray(B_bits, dtype=np.uint16)
    D = np.zeros((128, 64), dtype=np.float32)
    rc = lib.mma_selftest(A.ctypes.data, B.ctypes.data, D.ctypes.data, a_in_tmem)
    assert rc == 0, f"mma_selftest returned {rc}"
    return D


def test_single_mma_matches_numpy(lib):
    rng = np.random.default_rng(0)
    # small dyadic values: products and sums are exact in FP32
    A = rng.integers(-4, 5, size=(128, 32)) / 4.0
    Bm = rng.integers(-4, 5, size=(64, 32)) / 4.0
    D = _run(lib, kmajor_pack(A), kmajor_pack(Bm), 0)
    ref = A @ Bm.T
    assert np.array_equal(D, ref.astype(np.float32)), f"max diff {np.abs(D - ref).max()}"


def test_single_mma_with_a_from_tensor_memory(lib):
    rng = np.random.default_rng(1)
    A = rng.integers(-4, 5, size=(128, 32)) / 4.0
    Bm = rng.integers(-4, 5, size=(64, 32)) / 4.0
    D = _run(lib, A.astype(np.float16).view(np.uint16), kmajor_pack(Bm), 1)
    ref = A @ Bm.T
    assert np.array_equal(D, ref.astype(np.float32)), f"max diff {np.abs(D - ref).max()}"
