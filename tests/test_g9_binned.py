"""Material binning (nam_eval_binned, Sec. 7.3): queries with per-query
material ids, binned on the device, give bitwise the results of evaluating
each query with its own material alone; plus empty materials, one material,
the stochastic filter, FP8 and out-of-range ids."""
import numpy as np
import pytest

import workloads as W
from conftest import to_device

pytestmark = pytest.mark.gpu


def _materials(gctx, seed, k, precision=1, filt=0, W0=128, L=8):
    from paper_2305_02678_gb300 import binding as B
    rng = W.rng_streams(seed, 2 * k + 1)
    mats = []
    for j in range(k):
        pyr = W.make_pyramid(rng[j], W0, W0, L, dtype=np.float16)
        model = W.make_model(rng[k + j], (14, 64, 64, 3), (8, 16, 6))
        kw = {}
        if precision == B.NAM_PREC_FP8:
            kw["act_scale"] = np.array([0.004, 0.003, 0.0025], np.float32)
        mats.append(gctx.material(W0, W0, L, pyr, model["frame"], model["decoder"], precision=precision, filter=filt,
                                  **kw))
    return mats, rng[2 * k]


def _check_against_single(gctx, mats, dq, ids, n):
    import torch
    from paper_2305_02678_gb300 import binding as B
    out = torch.full((n, 3), -7.0, device="cuda")
    B.nam_eval_binned(gctx.h, [m.h for m in mats], dq, torch.from_numpy(ids).cuda(), n, out,
                      torch.cuda.current_stream())
    got = out.cpu().numpy()
    for k, m in enumerate(mats):
        sel = np.nonzero(ids == k)[0]
        if sel.size == 0:
            continue
        idx = torch.from_numpy(sel).cuda()
        sub = {f: t[idx].contiguous() for f, t in dq.items()}
        ref = m.eval(sub).cpu().numpy()
        assert np.array_equal(got[sel], ref), k
    return got


@pytest.mark.parametrize("n", [1, 127, 129, 5000, 65536])
def test_binned_equals_single_material(gctx, n):
    mats, rng = _materials(gctx, 71, 5)
    q = W.uniform_queries(rng, n, 7.0)
    ids = rng.integers(0, 5, n).astype(np.int32)
    _check_against_single(gctx, mats, to_device(q), ids, n)
    for m in mats:
        m.destroy()
    gctx.check()


def test_binned_empty_and_single_material(gctx):
    mats, rng = _materials(gctx, 72, 4)
    n = 3000
    q = W.uniform_queries(rng, n, 7.0)
    dq = to_device(q)
    ids = np.where(rng.random(n) < 0.5, 1, 3).astype(np.int32)   # materials 0 and 2 empty
    _check_against_single(gctx, mats, dq, ids, n)
    _check_against_single(gctx, mats[:1], dq, np.zeros(n, np.int32), n)
    for m in mats:
        m.destroy()
    gctx.check()


def test_binned_stochastic_and_fp8(gctx):
    from paper_2305_02678_gb300 import binding as B
    for prec, filt in ((B.NAM_PREC_F16, B.NAM_FILTER_STOCHASTIC), (B.NAM_PREC_FP8, B.NAM_FILTER_TRILINEAR)):
        mats, rng = _materials(gctx, 73, 3, precision=prec, filt=filt)
        n = 4097
        q = W.uniform_queries(rng, n, 7.0)
        ids = rng.integers(0, 3, n).astype(np.int32)
        _check_against_single(gctx, mats, to_device(q), ids, n)
        for m in mats:
            m.destroy()
    gctx.check()


def test_binned_out_of_range_ids(gctx):
    import torch
    from paper_2305_02678_gb300 import binding as B
    mats, rng = _materials(gctx, 74, 2)
    n = 1000
    q = W.uniform_queries(rng, n, 7.0)
    dq = to_device(q)
    ids = rng.integers(0, 2, n).astype(np.int32)
    ids[[5, 500]] = [7, -1]
    out = torch.full((n, 3), -7.0, device="cuda")
    B.nam_eval_binned(gctx.h, [m.h for m in mats], dq, torch.from_numpy(ids).cuda(), n, out,
                      torch.cuda.current_stream())
    with pytest.raises(B.NamError) as e:
        gctx.check()
    assert e.value.status == B.NAM_ERR_DEVICE_ASSERT
    got = out.cpu().numpy()
    assert np.all(got[[5, 500]] == -7.0)
    ok = np.ones(n, bool)
    ok[[5, 500]] = False
    for k, m in enumerate(mats):
        sel = np.nonzero(ok & (ids == k))[0]
        idx = torch.from_numpy(sel).cuda()
        ref = m.eval({f: t[idx].contiguous() for f, t in dq.items()}).cpu().numpy()
        assert np.array_equal(got[sel], ref)
    for m in mats:
        m.destroy()
    gctx.check()


def test_binned_many_materials(gctx):
    """257 materials (the plan kernel's search over material ranges, shared
    histograms of hundreds of entries), 20,000 queries, ids skewed so that
    some materials get one query and some none."""
    mats, rng = _materials(gctx, 75, 257, W0=16, L=4)
    n = 20000
    q = W.uniform_queries(rng, n, 3.0)
    ids = np.minimum(rng.geometric(0.02, n) - 1, 256).astype(np.int32)
    _check_against_single(gctx, mats, to_device(q), ids, n)
    for m in mats:
        m.destroy()
    gctx.check()
