"""FP8 (E4M3) decoder path (beyond the paper, which stops at FP16 parameters,
Sec. 5.2): the hidden -> hidden layers -- most of the decoder's MACs -- have
E4M3 weights with a power-of-two per-layer scale; their input activations
enter as two E4M3 code sets (hi = E4M3(x / s_a), lo = E4M3(x / s_a - hi), s_a
the power of two above the calibrated max |input| / 448), FP32 accumulation;
the frame MLP and the first and last decoder layers as in the FP16 path.

Parity: against the oracle evaluating the same parameter values (params=
"fp8": those E4M3 weights, binary16 elsewhere) with FP64 activations, within
the stated FP8 bound 3e-2 at the maximum (kappa <= 50; conditioning-aware
beyond).  The error against the FP32 masters is reported."""
import numpy as np
import pytest

import workloads as W
from conftest import to_device

pytestmark = pytest.mark.gpu

TOL_F8 = 3e-2


@pytest.fixture(scope="module")
def w3s():
    return W.workload(3, scale=1 / 32)   # 3840 x 68 = 261,120 warp queries


@pytest.fixture(scope="module")
def calib(oracle, w3s):
    """Activation scales from the oracle (FP64 forward of the masters) over the
    calibration batch."""
    m = w3s["model"]
    om = oracle.Model(w3s["W0"], w3s["H0"], w3s["L"], w3s["pyramid"], m["frame"], m["decoder"])
    amax = oracle.decoder_input_absmax(om, W.calibration_queries(3))
    return np.where(amax > 0, amax / 448.0, 1.0).astype(np.float32)


def test_fp8_calibration_matches_oracle_ranges(gctx, oracle, w3s, calib):
    from paper_2305_02678_gb300 import binding as B
    m = w3s["model"]
    mat = gctx.material(w3s["W0"], w3s["H0"], w3s["L"], w3s["pyramid"], m["frame"], m["decoder"],
                        precision=B.NAM_PREC_F16)
    cq = W.calibration_queries(3)
    got = B.nam_fp8_calibrate(gctx.h, mat.h, to_device(cq), len(cq["u"]))[:3]
    print("scales gpu", got, "oracle", calib)
    assert np.allclose(got, calib, rtol=1e-5, atol=0)
    mat.destroy()


def _fp8_material(ctx, w, scales, **kw):
    from paper_2305_02678_gb300 import binding as B
    m = w["model"]
    return ctx.material(w["W0"], w["H0"], w["L"], w["pyramid"], m["frame"], m["decoder"], precision=B.NAM_PREC_FP8,
                        act_scale=scales, **kw)


def _check_fp8(oracle, w, scales, g, filt=0, addr=0, label="fp8", q=None):
    m = w["model"]
    q = w["queries"] if q is None else q
    om = oracle.Model(w["W0"], w["H0"], w["L"], w["pyramid"], m["frame"], m["decoder"], filter=filt, address=addr,
                      params="fp8")
    o = oracle.eval(om, q)
    kappa = oracle.frame_condition(om, q)
    ok, st = oracle.parity(g, o, kappa, TOL_F8, gain=oracle.band_gain(om, q, kappa))
    print(f"{label}: vs oracle (E4M3 hidden weights, FP64 activations) max {st['max_rel']:.3e} "
          f"(well-conditioned {st['max_rel_well_conditioned']:.3e}) mean {st['mean_rel']:.3e}, "
          f"ill-conditioned {st['ill_conditioned']}/{st['n']}")
    assert ok, st
    assert st["max_rel_well_conditioned"] <= TOL_F8
    return om


def test_fp8_sweep_workload(gctx, oracle, w3s, calib):
    """The 4K sweep's generator (3840 wide), 261k queries, FP8 vs oracle."""
    mat = _fp8_material(gctx, w3s, calib)
    g = mat.eval(to_device(w3s["queries"])).cpu().numpy()
    info = mat.info
    mat.destroy()
    gctx.check()
    _check_fp8(oracle, w3s, calib, g, label="fp8 3840x68")
    m = w3s["model"]
    master = oracle.eval(oracle.Model(w3s["W0"], w3s["H0"], w3s["L"], w3s["pyramid"], m["frame"], m["decoder"]),
                         w3s["queries"])
    e2 = oracle.relative_error(g, master)
    print(f"fp8 vs FP32-master oracle: max {e2[0]:.3e} mean {e2[1]:.3e}")
    print("weight scales", list(info.fp8_weight_scale)[:3])
    # the weight scale the library reports for the E4M3 layer is the oracle's;
    # the FP16 layers report none
    sc = list(info.fp8_weight_scale)[:3]
    assert sc[1] == oracle.quantize_e4m3_layer(m["decoder"][1][0])[0]
    assert sc[0] == 0.0 and sc[2] == 0.0


@pytest.mark.parametrize("filt", [0, 1])
@pytest.mark.parametrize("addr", [0, 1])
def test_fp8_filters_and_addressing(gctx, oracle, w3s, calib, filt, addr):
    q = W.slice_queries(w3s["queries"], 0, 40000)
    mat = _fp8_material(gctx, w3s, calib, filter=filt, address=addr)
    g = mat.eval(to_device(q)).cpu().numpy()
    mat.destroy()
    _check_fp8(oracle, w3s, calib, g, filt=filt, addr=addr, label=f"fp8 filt={filt} addr={addr}", q=q)


@pytest.mark.parametrize("H,NH", [(16, 2), (32, 2), (64, 2), (64, 3)])
@pytest.mark.parametrize("frame", ["none", "mlp", "paper"])
@pytest.mark.parametrize("latent", ["f16", "f32"])
def test_fp8_shapes(gctx, oracle, H, NH, frame, latent):
    from paper_2305_02678_gb300 import binding as B
    rng = W.rng_streams(500 + H + 7 * NH + 2 * len(frame), 3)
    W0 = H0 = 256
    L = 9
    pyr = W.make_pyramid(rng[0], W0, H0, L, dtype=np.float16 if latent == "f16" else np.float32)
    fw = {"none": None, "mlp": (8, 16, 6), "paper": (8, 12)}[frame]
    model = W.make_model(rng[1], (20 if frame == "paper" else 14,) + (H,) * NH + (3,), fw)
    q = W.uniform_queries(rng[2], 20000, 8.0)
    w = dict(W0=W0, H0=H0, L=L, pyramid=pyr, model=model, queries=q)
    om = oracle.Model(W0, H0, L, pyr, model["frame"], model["decoder"])
    amax = oracle.decoder_input_absmax(om, W.uniform_queries(W.rng_streams(900 + H, 1)[0], 65536, 8.0))
    scales = np.where(amax > 0, amax / 448.0, 1.0).astype(np.float32)
    mat = gctx.material(W0, H0, L, pyr, model["frame"], model["decoder"], precision=B.NAM_PREC_FP8, act_scale=scales)
    g = mat.eval(to_device(q)).cpu().numpy()
    mat.destroy()
    _check_fp8(oracle, w, scales, g, label=f"fp8 {NH}x{H} frame={frame} {latent}")


def test_fp8_ragged_and_multi(gctx, oracle, w3s, calib):
    """Ragged counts through nam_eval, and an FP8 multi-material launch gives
    each item what its own single-material launch gives (bitwise)."""
    import torch
    from paper_2305_02678_gb300 import binding as B
    mat = _fp8_material(gctx, w3s, calib)
    dq = to_device(W.slice_queries(w3s["queries"], 0, 5000))
    full = mat.eval(dq)
    for n in (1, 127, 129, 4097):
        sub = {k: v[:n] for k, v in dq.items()}
        assert torch.equal(mat.eval(sub), full[:n])
    m2 = w3s["model"]
    rng = W.rng_streams(77, 2)
    other = gctx.material(w3s["W0"], w3s["H0"], w3s["L"], W.make_pyramid(rng[0], 2048, 2048, 12, dtype=np.float16),
                          m2["frame"], m2["decoder"], precision=B.NAM_PREC_FP8, act_scale=calib)
    ref_other = other.eval(dq)
    items = [(0, 128, 0), (128, 100, 1), (228, 128, 0), (356, 4644, 1)]
    out = torch.empty_like(full)
    B.nam_eval_multi(gctx.h, [mat.h, other.h], dq, items, out, torch.cuda.current_stream())
    torch.cuda.synchronize()
    for s, c, k in items:
        ref = full if k == 0 else ref_other
        assert torch.equal(out[s:s + c], ref[s:s + c])
    mat.destroy()
    other.destroy()
    gctx.check()


def test_fp8_rejects_bad_scales(gctx, w3s):
    from paper_2305_02678_gb300 import binding as B
    for bad in (None, [1.0, 0.0, 1.0], [1.0, float("nan"), 1.0]):
        with pytest.raises(B.NamError):
            _fp8_material(gctx, w3s, None if bad is None else np.array(bad, dtype=np.float32))
