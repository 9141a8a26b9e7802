"""One tcgen05 MMA in isolation: shared-memory descriptors, instruction
descriptor and TMEM read-back conventions that every tensor-core kernel
relies on.  Runs before the evaluation tests."""
import numpy as np
import pytest

from conftest import kmajor_pack

pytestmark = pytest.mark.gpu


def test_single_mma_matches_numpy(gctx):
    from paper_2305_02678_gb300 import binding as B
    rng = np.random.default_rng(0)
    # small dyadic values: products and sums are exact in FP32
    A = rng.integers(-4, 5, size=(128, 32)) / 4.0
    Bm = rng.integers(-4, 5, size=(64, 32)) / 4.0
    D = B.nam_debug_mma_selftest(gctx.h, kmajor_pack(A), kmajor_pack(Bm))
    ref = A @ Bm.T
    assert np.array_equal(D, ref.astype(np.float32)), f"max diff {np.abs(D - ref).max()}"


def test_single_mma_with_a_from_tensor_memory(gctx):
    from paper_2305_02678_gb300 import binding as B
    rng = np.random.default_rng(1)
    A = rng.integers(-4, 5, size=(128, 32)) / 4.0
    Bm = rng.integers(-4, 5, size=(64, 32)) / 4.0
    D = B.nam_debug_mma_selftest_ts(gctx.h, A.astype(np.float16).view(np.uint16), kmajor_pack(Bm))
    ref = A @ Bm.T
    assert np.array_equal(D, ref.astype(np.float32)), f"max diff {np.abs(D - ref).max()}"
