import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a) and the built libnam.so")


@pytest.fixture(scope="session")
def oracle():
    import oracle.oracle as O
    O.build()
    return O


@pytest.fixture(scope="session")
def gctx():
    """A libnam context on cuda:0 shared by the GPU tests."""
    from paper_2305_02678_gb300 import Context, _build
    _build.build()
    ctx = Context(0)
    yield ctx
    ctx.close()


def to_device(q):
    import torch
    return {k: torch.from_numpy(v).cuda() for k, v in q.items()}


def kmajor_pack(M):
    """binary16 bits of an R x K matrix in the canonical no-swizzle K-major
    core-matrix layout: element (r, k) at (k/8)*R*16 + r*16 + (k%8)*2 bytes."""
    import numpy as np
    R, K = M.shape
    out = np.zeros(R * K, dtype=np.uint16)
    bits = M.astype(np.float16).view(np.uint16)
    for k in range(K):
        for r in range(R):
            out[((k // 8) * R * 16 + r * 16 + (k % 8) * 2) // 2] = bits[r, k]
    return out
