"""nam_train_step_noalloc: the training step for callers that may not
allocate device memory (its per-batch buffers live in the library's static
device array).  It must give what nam_train_step gives: two identical
trainable materials, steps in a row on the same batches (the last one at the
largest batch the static array holds), one through each entry point.  Collected last on purpose (file name), and independent of every
other test's state, so it passes alone in a fresh process and after the rest."""
import numpy as np
import pytest

import workloads as W
from conftest import to_device

pytestmark = pytest.mark.gpu


class _DevArray:
    def __init__(self, ptr, n):
        self.__cuda_array_interface__ = {"shape": (n,), "typestr": "<f4", "data": (ptr, False), "version": 3}


def test_noalloc_training_step_matches_allocating_step():
    import torch
    from paper_2305_02678_gb300 import Context, _build
    _build.build()
    from paper_2305_02678_gb300 import binding as B
    rng = W.rng_streams(404, 4)
    W0 = H0 = 128
    L = 8
    pyr = W.make_pyramid(rng[0], W0, H0, L, dtype=np.float32)
    model = W.make_model(rng[1], (14, 64, 64, 3), (8, 16, 6))
    target = W.ProceduralBRDF(rng[2])
    with Context(0) as ctx:
        ref = ctx.material(W0, H0, L, pyr, model["frame"], model["decoder"], precision=B.NAM_PREC_F32, trainable=True)
        nal = ctx.material(W0, H0, L, pyr, model["frame"], model["decoder"], precision=B.NAM_PREC_F32, trainable=True)
        s = torch.cuda.current_stream()
        # two ordinary steps, then one at the largest batch the static array
        # holds (its last slot in use)
        for step, n in ((1, 20000), (2, 20000), (3, B.NAM_NOALLOC_TRAIN_MAX_QUERIES)):
            q = W.uniform_queries(rng[3], n, 7.0)
            y = torch.from_numpy(W.target_rgb(target, q)).cuda()
            dq = to_device(q)
            l_ref = B.nam_train_step(ctx.h, ref.h, dq, y, n, step=step, stream=s)
            l_nal = B.nam_train_step_noalloc(ctx.h, nal.h, dq, y, n, step=step, stream=s)
            assert np.isfinite(l_ref) and np.isfinite(l_nal)
            assert abs(l_ref - l_nal) <= 1e-5 * abs(l_ref), (step, l_ref, l_nal)
        torch.cuda.synchronize()
        pr, zr = ref.params()
        pn, zn = nal.params()
        P = lambda p, m: torch.as_tensor(_DevArray(p, m), device="cuda")
        a, b = P(pr, ref.info.n_params), P(pn, nal.info.n_params)
        # the allocating step fuses forward and loss into its backward kernel:
        # the two differ in FP32 summation order only
        assert torch.allclose(a, b, rtol=1e-4, atol=1e-6), (a - b).abs().max().item()
        za, zb = P(zr, ref.info.texels * 8), P(zn, nal.info.texels * 8)
        assert torch.allclose(za, zb, rtol=1e-4, atol=1e-6), (za - zb).abs().max().item()
        # the size limit is enforced before anything runs
        big = B.NAM_NOALLOC_TRAIN_MAX_QUERIES + 1
        qb = {k: torch.zeros(big, device="cuda") for k in B.QUERY_FIELDS if k != "xi"}
        with pytest.raises(B.NamError) as e:
            B.nam_train_step_noalloc(ctx.h, nal.h, qb, torch.zeros((big, 3), device="cuda"), big, stream=s)
        assert e.value.status == B.NAM_ERR_INVALID_ARG
        ctx.check()
