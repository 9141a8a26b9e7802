"""The paper's own decoder shapes on the GPU: its frame form (one linear layer
8 -> 12, two normalised non-orthogonal frames, 20-input decoder; Sec. 4.2,
Eq. 4, Sec. 9) and its three decoder sizes (2 x 16, 2 x 32, 3 x 64 hidden
units; Sec. 8), in FP32 and FP16, against the oracle with the same tolerances
as the benchmark's shape (1e-5 FP32, 2e-3 FP16, both against the oracle with
the same parameter values and FP64 activations; conditioning-aware beyond
kappa = 50)."""
import numpy as np
import pytest

import workloads as W
from conftest import to_device

pytestmark = pytest.mark.gpu

SIZES = [(16, 2), (32, 2), (64, 3)]


def _setup(seed, H, NH, frame, n=20000, latent="f16"):
    rng = W.rng_streams(seed, 3)
    W0 = H0 = 256
    L = 9
    pyr = W.make_pyramid(rng[0], W0, H0, L, dtype=np.float16 if latent == "f16" else np.float32)
    fw = {"paper": (8, 12), "mlp": (8, 16, 6), "none": None}[frame]
    nin = 20 if frame == "paper" else 14
    model = W.make_model(rng[1], (nin,) + (H,) * NH + (3,), fw)
    q = W.uniform_queries(rng[2], n, 8.0)
    return W0, H0, L, pyr, model, q


def _check(oracle, g, om, q, tol, label):
    o = oracle.eval(om, q)
    kappa = oracle.frame_condition(om, q)
    ok, st = oracle.parity(g, o, kappa, tol, gain=oracle.band_gain(om, q, kappa))
    print(f"{label}: max {st['max_rel']:.3e} (well-conditioned {st['max_rel_well_conditioned']:.3e}), "
          f"ill-conditioned {st['ill_conditioned']}/{st['n']}")
    assert ok, st


@pytest.mark.parametrize("H,NH", SIZES)
@pytest.mark.parametrize("frame", ["paper", "mlp", "none"])
def test_fp32_paper_sizes(gctx, oracle, H, NH, frame):
    from paper_2305_02678_gb300 import binding as B
    W0, H0, L, pyr, model, q = _setup(81 + H + NH, H, NH, frame)
    mat = gctx.material(W0, H0, L, pyr, model["frame"], model["decoder"], precision=B.NAM_PREC_F32)
    g = mat.eval(to_device(q)).cpu().numpy()
    mat.destroy()
    om = oracle.Model(W0, H0, L, pyr, model["frame"], model["decoder"])
    _check(oracle, g, om, q, 1e-5, f"fp32 {frame} {NH}x{H}")


@pytest.mark.parametrize("H,NH", SIZES)
@pytest.mark.parametrize("frame", ["paper", "mlp", "none"])
@pytest.mark.parametrize("latent", ["f16", "f32"])
def test_fp16_paper_sizes(gctx, oracle, H, NH, frame, latent):
    from paper_2305_02678_gb300 import binding as B
    W0, H0, L, pyr, model, q = _setup(91 + H + NH, H, NH, frame, latent=latent)
    mat = gctx.material(W0, H0, L, pyr, model["frame"], model["decoder"], precision=B.NAM_PREC_F16)
    g = mat.eval(to_device(q)).cpu().numpy()
    mat.destroy()
    gctx.check()
    om = oracle.Model(W0, H0, L, pyr, model["frame"], model["decoder"], params="fp16")
    _check(oracle, g, om, q, 2e-3, f"fp16 {frame} {NH}x{H} {latent}")


def test_paper_form_multi_material_and_ragged(gctx):
    import torch
    from paper_2305_02678_gb300 import binding as B
    W0, H0, L, pyr, model, q = _setup(95, 64, 3, "paper", n=5000)
    rng = W.rng_streams(96, 2)
    model2 = W.make_model(rng[0], (20, 64, 64, 64, 3), (8, 12))
    pyr2 = W.make_pyramid(rng[1], W0, H0, L, dtype=np.float16)
    a = gctx.material(W0, H0, L, pyr, model["frame"], model["decoder"])
    b = gctx.material(W0, H0, L, pyr2, model2["frame"], model2["decoder"])
    dq = to_device(q)
    ra, rb = a.eval(dq), b.eval(dq)
    for n in (1, 127, 129, 4097):
        assert torch.equal(a.eval({k: v[:n] for k, v in dq.items()}), ra[:n])
    items = [(0, 300, 1), (300, 128, 0), (428, 4572, 1)]
    out = torch.empty_like(ra)
    B.nam_eval_multi(gctx.h, [a.h, b.h], dq, items, out, torch.cuda.current_stream())
    torch.cuda.synchronize()
    for s, c, k in items:
        assert torch.equal(out[s:s + c], (ra if k == 0 else rb)[s:s + c])
    a.destroy()
    b.destroy()
    gctx.check()


def test_unsupported_combinations_fail_cleanly(gctx):
    from paper_2305_02678_gb300 import binding as B
    W0, H0, L, pyr, model, q = _setup(97, 64, 2, "paper", n=10)
    with pytest.raises(B.NamError):   # FP8 needs its activation scales
        gctx.material(W0, H0, L, pyr, model["frame"], model["decoder"], precision=B.NAM_PREC_FP8)
    pyr32 = pyr.astype(np.float32)
    with pytest.raises(B.NamError):   # training needs the frame MLP form
        gctx.material(W0, H0, L, pyr32, model["frame"], model["decoder"], precision=B.NAM_PREC_F32, trainable=True)
    _, _, _, _, m32, _ = _setup(98, 32, 3, "mlp", n=10)
    with pytest.raises(B.NamError):   # three hidden layers need H = 64
        gctx.material(W0, H0, L, pyr, m32["frame"], m32["decoder"])
