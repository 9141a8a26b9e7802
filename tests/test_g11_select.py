"""Per-tile selection between code paths (nam_eval_select, Sec. 7.1).  A
tile of 128 queries with at most NAM_SELECT_MAX_PASSES distinct materials
(one) runs as one tensor-core pass per material; the queries of tiles with
more are binned by material (the SER analogue, Sec. 7.3) and run in
material-coherent chunks.  Either way every query must be bitwise nam_eval
on its material, so the whole output equals nam_eval_binned's; one case per
precision is also graded against the FP64 oracle (FP16 bound 2e-3, FP8
3e-2, conditioning-aware beyond kappa = 50).  Plus ragged sizes, coherent,
few-material and many-material tiles, the paper's decoder shapes, the
stochastic filter, the cosine factor and out-of-range ids."""
import numpy as np
import pytest

import workloads as W
from conftest import to_device

pytestmark = pytest.mark.gpu

TOL = {1: 2e-3, 2: 3e-2}


def _materials(gctx, oracle, seed, k, precision=1, filt=0, W0=128, L=8, H=64, NH=2, frame="mlp", cos=False):
    from paper_2305_02678_gb300 import binding as B
    rng = W.rng_streams(seed, 2 * k + 1)
    fw = {"paper": (8, 12), "mlp": (8, 16, 6), "none": None}[frame]
    nin = 20 if frame == "paper" else 14
    mats, models = [], []
    for j in range(k):
        pyr = W.make_pyramid(rng[j], W0, W0, L, dtype=np.float16)
        model = W.make_model(rng[k + j], (nin,) + (H,) * NH + (3,), fw)
        kw = {}
        if precision == B.NAM_PREC_FP8:
            # calibrated input scales of the decoder layers (max |input| / 448)
            om = oracle.Model(W0, W0, L, pyr, model["frame"], model["decoder"], filter=filt)
            amax = oracle.decoder_input_absmax(om, W.uniform_queries(np.random.default_rng(seed + j), 4096, 6.0))
            kw["act_scale"] = np.where(amax > 0, amax / 448.0, 1.0).astype(np.float32)
        mats.append(gctx.material(W0, W0, L, pyr, model["frame"], model["decoder"], precision=precision,
                                  filter=filt, **kw))
        params = "fp8" if precision == B.NAM_PREC_FP8 else "fp16"
        models.append(oracle.Model(W0, W0, L, pyr, model["frame"], model["decoder"], filter=filt, params=params,
                                   out_cosine=cos))
    return mats, models, rng[2 * k]


def _tile_ids(rng, n, k, mixed_frac, many_frac=0.0):
    """One material per 128-query tile; in a fraction of the tiles 1 to 40
    queries take another material, in another fraction every query draws
    its own."""
    tiles = (n + 127) // 128
    ids = np.repeat(rng.integers(0, k, tiles), 128)[:n].copy()
    u = rng.random(tiles)
    for t in np.nonzero(u < mixed_frac)[0]:
        lo, hi = 128 * t, min(n, 128 * t + 128)
        m = int(rng.integers(1, 41))
        ids[rng.integers(lo, hi, m)] = rng.integers(0, k, m)
    for t in np.nonzero((u >= mixed_frac) & (u < mixed_frac + many_frac))[0]:
        lo, hi = 128 * t, min(n, 128 * t + 128)
        ids[lo:hi] = rng.integers(0, k, hi - lo)
    return ids.astype(np.int32)


def _on_passes(ids, nmat, max_passes):
    """Per query: does its tile run as tensor-core passes (at most
    max_passes distinct valid materials), rather than through binning?"""
    n = len(ids)
    out = np.zeros(n, bool)
    for t in range((n + 127) // 128):
        s = ids[128 * t:128 * t + 128]
        out[128 * t:128 * t + 128] = np.unique(s[(s >= 0) & (s < nmat)]).size <= max_passes
    return out


def _run(gctx, mats, dq, ids, n, flags=0):
    import torch
    from paper_2305_02678_gb300 import binding as B
    out = torch.full((n, 3), -7.0, device="cuda")
    B.nam_eval_select(gctx.h, [m.h for m in mats], dq, torch.from_numpy(ids).cuda(), n, out,
                      torch.cuda.current_stream(), flags)
    return out.cpu().numpy()


def _check(gctx, oracle, mats, models, q, ids, n, flags=0, label="", precision=None):
    """Every valid query bitwise nam_eval on its material, the output
    bitwise nam_eval_binned's; with `precision`, also graded against the
    oracle."""
    import torch
    from paper_2305_02678_gb300 import binding as B
    dq = to_device(q)
    got = _run(gctx, mats, dq, ids, n, flags)
    gctx.check()
    tc = _on_passes(ids, len(mats), B.NAM_SELECT_MAX_PASSES)
    for k, (m, om) in enumerate(zip(mats, models)):
        sel = np.nonzero(ids == k)[0]
        if sel.size == 0:
            continue
        idx = torch.from_numpy(sel).cuda()
        ref = m.eval({f: t[idx].contiguous() for f, t in dq.items()}, flags=flags).cpu().numpy()
        assert np.array_equal(got[sel], ref), (label, k)
        if precision is not None:
            sq = {f: v[sel] for f, v in q.items()}
            kappa = oracle.frame_condition(om, sq)
            ok, st = oracle.parity(got[sel], oracle.eval(om, sq), kappa, TOL[precision],
                                   gain=oracle.band_gain(om, sq, kappa))
            assert ok, (label, k, st)
    binned = torch.full((n, 3), -7.0, device="cuda")
    B.nam_eval_binned(gctx.h, [m.h for m in mats], dq, torch.from_numpy(ids).cuda(), n, binned,
                      torch.cuda.current_stream(), flags)
    assert np.array_equal(got, binned.cpu().numpy()), label
    print(f"{label}: {int(tc.sum())} queries on tensor-core passes, {int((~tc).sum())} binned")
    return got, tc


@pytest.mark.parametrize("n", [1, 127, 129, 5000, 65536])
def test_select_tiles(gctx, oracle, n):
    mats, models, rng = _materials(gctx, oracle, 101, 12, W0=64, L=7)
    q = W.uniform_queries(rng, n, 6.0)
    ids = _tile_ids(rng, n, 12, 0.3, 0.2)
    _, tc = _check(gctx, oracle, mats, models, q, ids, n, label=f"n={n}", precision=1 if n == 5000 else None)
    if n >= 5000:
        assert tc.any() and not tc.all()
    for m in mats:
        m.destroy()
    gctx.check()


def test_select_all_coherent_few_and_many(gctx, oracle):
    import torch
    from paper_2305_02678_gb300 import binding as B
    mats, models, rng = _materials(gctx, oracle, 102, 12, W0=64, L=7)
    n = 4000
    q = W.uniform_queries(rng, n, 6.0)
    dq = to_device(q)
    # one material: the whole batch bitwise nam_eval
    got = _run(gctx, mats[:1], dq, np.zeros(n, np.int32), n)
    assert np.array_equal(got, mats[0].eval(dq).cpu().numpy())
    # three materials per query at random: three passes per tile if the
    # pass limit allows, else every tile binned
    ids = rng.integers(0, 3, n).astype(np.int32)
    _, tc = _check(gctx, oracle, mats, models, q, ids, n, label="3 per tile")
    assert tc.all() == (3 <= B.NAM_SELECT_MAX_PASSES) and tc.any() == (3 <= B.NAM_SELECT_MAX_PASSES)
    # exactly NAM_SELECT_MAX_PASSES materials per tile: still passes; one more: binned
    for k, on_passes in ((B.NAM_SELECT_MAX_PASSES, True), (B.NAM_SELECT_MAX_PASSES + 1, False)):
        ids = (np.arange(n) % k).astype(np.int32)
        _, tc = _check(gctx, oracle, mats, models, q, ids, n, label=f"{k} per tile")
        assert tc.all() == on_passes and tc.any() == on_passes
    # twelve materials per query at random: every tile binned
    ids = rng.integers(0, 12, n).astype(np.int32)
    _, tc = _check(gctx, oracle, mats, models, q, ids, n, label="12 per tile")
    assert not tc.any()
    # a mixed batch of all three kinds of tile
    ids = _tile_ids(rng, n, 12, 0.5, 0.2)
    _, tc = _check(gctx, oracle, mats, models, q, ids, n, label="mixed")
    assert tc.any() and not tc.all()
    for m in mats:
        m.destroy()
    gctx.check()


@pytest.mark.parametrize("H,NH,frame", [(16, 2, "none"), (32, 2, "mlp"), (64, 3, "paper"), (64, 2, "paper")])
def test_select_decoder_shapes(gctx, oracle, H, NH, frame):
    mats, models, rng = _materials(gctx, oracle, 103 + H + NH, 10, H=H, NH=NH, frame=frame, W0=64, L=7)
    n = 6000
    q = W.uniform_queries(rng, n, 6.0)
    _check(gctx, oracle, mats, models, q, _tile_ids(rng, n, 10, 0.4, 0.3), n, label=f"{NH}x{H} {frame}")
    for m in mats:
        m.destroy()
    gctx.check()


def test_select_fp8_stochastic_cosine(gctx, oracle):
    from paper_2305_02678_gb300 import binding as B
    for prec, filt, cos in ((B.NAM_PREC_FP8, B.NAM_FILTER_TRILINEAR, False),
                            (B.NAM_PREC_F16, B.NAM_FILTER_STOCHASTIC, True),
                            (B.NAM_PREC_FP8, B.NAM_FILTER_STOCHASTIC, True)):
        mats, models, rng = _materials(gctx, oracle, 104, 10, precision=prec, filt=filt, cos=cos, W0=64, L=7)
        n = 4097
        q = W.uniform_queries(rng, n, 6.0)
        _check(gctx, oracle, mats, models, q, _tile_ids(rng, n, 10, 0.4, 0.3), n,
               flags=B.NAM_OUT_COSINE if cos else 0, label=f"precision {prec} filter {filt} cosine {cos}",
               precision=prec)
        for m in mats:
            m.destroy()
    gctx.check()


def test_select_out_of_range_ids(gctx, oracle):
    import torch
    from paper_2305_02678_gb300 import binding as B
    mats, models, rng = _materials(gctx, oracle, 105, 10, W0=64, L=7)
    n = 1000
    q = W.uniform_queries(rng, n, 6.0)
    ids = _tile_ids(rng, n, 10, 0.0)
    ids[256:384] = rng.integers(0, 10, 128)   # tile 2: binned
    ids[[5, 300, 500, 999]] = [7 + 10, -1, 10, -5]
    dq = to_device(q)
    got = _run(gctx, mats, dq, ids, n)
    with pytest.raises(B.NamError) as e:
        gctx.check()
    assert e.value.status == B.NAM_ERR_DEVICE_ASSERT
    bad = np.array([5, 300, 500, 999])
    assert np.all(got[bad] == -7.0)
    ok = np.ones(n, bool)
    ok[bad] = False
    tc = _on_passes(ids, 10, B.NAM_SELECT_MAX_PASSES)
    assert tc[5] and not tc[300] and tc[500]
    for k, (m, om) in enumerate(zip(mats, models)):
        sel = np.nonzero(ok & (ids == k))[0]
        if sel.size:
            idx = torch.from_numpy(sel).cuda()
            ref = m.eval({f: t[idx].contiguous() for f, t in dq.items()}).cpu().numpy()
            assert np.array_equal(got[sel], ref)
    for m in mats:
        m.destroy()
    gctx.check()
