"""A device-side wait that runs out (nam_init's wait_timeout_ns; the library's
NAM_ERR_TIMEOUT): no GPU fault, hang or trap is involved.

A context whose limit (1 ns) is shorter than any MMA or bulk copy makes the
tensor-core kernels' steady-state waits give up; each kernel then records the
timeout in the context's error word, waits for its own MMAs and copies with
the fixed drain limit, frees its TMEM and returns.  The test checks that the
status comes back as NAM_ERR_TIMEOUT, that a second check is clean (the word
is cleared), and that a context with the default limit evaluates the same
queries correctly afterwards (the GPU is still usable: no TMEM was leaked on
any SM, since a later kernel allocates all 512 columns of every SM)."""
import numpy as np
import pytest

import workloads as W
from conftest import to_device

pytestmark = pytest.mark.gpu


def _workload():
    rng = W.rng_streams(1301, 3)
    W0 = H0 = 512
    L = 10
    pyr = W.make_pyramid(rng[0], W0, H0, L, dtype=np.float16)
    model = W.make_model(rng[1], (14, 64, 64, 3), (8, 16, 6))
    q = W.uniform_queries(rng[2], 300000, 9.0)
    return W0, H0, L, pyr, model, q


@pytest.mark.parametrize("precision", [1, 2])
def test_short_wait_limit_reports_timeout_and_gpu_stays_usable(oracle, precision):
    from paper_2305_02678_gb300 import Context
    from paper_2305_02678_gb300 import binding as B
    W0, H0, L, pyr, model, q = _workload()
    dq = to_device(q)
    kw = {}
    if precision == B.NAM_PREC_FP8:
        om = oracle.Model(W0, H0, L, pyr, model["frame"], model["decoder"])
        amax = oracle.decoder_input_absmax(om, W.slice_queries(q, 0, 20000))
        kw["act_scale"] = np.where(amax > 0, amax / 448.0, 1.0).astype(np.float32)
    with Context(0, wait_timeout_ns=1) as short:
        mat = short.material(W0, H0, L, pyr, model["frame"], model["decoder"], precision=precision, **kw)
        for _ in range(3):
            mat.eval(dq)
        with pytest.raises(B.NamError) as e:
            short.check()
        assert e.value.status == B.NAM_ERR_TIMEOUT
        short.check()  # the error word was cleared (no launch since)
        mat.destroy()
    with Context(0) as ok:
        mat = ok.material(W0, H0, L, pyr, model["frame"], model["decoder"], precision=precision, **kw)
        g = mat.eval(dq).cpu().numpy()
        ok.check()
        mat.destroy()
    n = 20000
    params = "fp16" if precision == B.NAM_PREC_F16 else "fp8"
    om = oracle.Model(W0, H0, L, pyr, model["frame"], model["decoder"], params=params)
    o = oracle.eval(om, W.slice_queries(q, 0, n))
    err = oracle.relative_error(g[:n], o)[0]
    assert np.isfinite(g).all()
    assert err <= (2e-3 if precision == B.NAM_PREC_F16 else 3e-2)


def test_sampler_short_wait_limit_reports_timeout(oracle):
    """The same for the tensor-core importance sampler: a 1 ns limit gives
    NAM_ERR_TIMEOUT, and a context with the default limit then matches the
    oracle's densities."""
    import torch
    from paper_2305_02678_gb300 import Context
    from paper_2305_02678_gb300 import binding as B
    W0, H0, L, pyr, model, q = _workload()
    sampler = W.make_mlp(W.rng_streams(1302, 1)[0], (11, 32, 32, 32, 9))
    dq = to_device(q)
    n = len(q["u"])
    out = torch.empty(n, device="cuda")
    with Context(0, wait_timeout_ns=1) as short:
        mat = short.material(W0, H0, L, pyr, model["frame"], model["decoder"], sampler=sampler)
        for _ in range(3):
            B.nam_sample_pdf(short.h, mat.h, dq, n, out)
        with pytest.raises(B.NamError) as e:
            short.check()
        assert e.value.status == B.NAM_ERR_TIMEOUT
        mat.destroy()
    with Context(0) as ok:
        mat = ok.material(W0, H0, L, pyr, model["frame"], model["decoder"], sampler=sampler)
        B.nam_sample_pdf(ok.h, mat.h, dq, n, out)
        ok.check()
        g = out[:20000].cpu().numpy().astype(np.float64)
        mat.destroy()
    o = oracle.sampler_pdf(oracle.Model(W0, H0, L, pyr, model["frame"], model["decoder"]), sampler,
                           W.slice_queries(q, 0, 20000))
    rel = np.abs(g - o) / np.maximum(np.abs(o), 1e-3 * np.median(o))
    assert np.isfinite(g).all() and np.percentile(rel, 99) < 1e-4
