"""The optional albedo head on the GPU (the paper's albedo inference: the
decoder's extra RGB triplet approximates the directional albedo of Eq. 2 and
is trained with an L2 loss against one-sample estimates).  Evaluation in
FP32, FP16 and FP8 against the oracle's six-output decoder with the
tolerances of the RGB path (1e-5 FP32, 2e-3 FP16 and 3e-2 FP8 against the
oracle with the same parameter values and FP64 activations); the RGB of a
material
with the head is nam_eval's; reverse mode with [n][6] output gradients; the
fused training step's loss and update direction against the oracle; a fit
of the head to the procedural material's albedo; refused combinations."""
import numpy as np
import pytest

import workloads as W
from conftest import to_device

pytestmark = pytest.mark.gpu

TOL_F32, TOL_F16, TOL_F8 = 1e-5, 2e-3, 3e-2


def _setup(seed, n=20000, H=64, NH=2, frame="mlp", latent=np.float16, W0=128, L=8):
    rng = W.rng_streams(seed, 3)
    pyr = W.make_pyramid(rng[0], W0, W0, L, dtype=latent)
    fw = {"paper": (8, 12), "mlp": (8, 16, 6), "none": None}[frame]
    nin = 20 if frame == "paper" else 14
    model = W.make_model(rng[1], (nin,) + (H,) * NH + (6,), fw)
    q = W.uniform_queries(rng[2], n, float(L - 1))
    return W0, L, pyr, model, q


def _parity(oracle, g, o, kappa, tol, label):
    """RGB and albedo channel groups, each against its own RMS scale."""
    for name, sl in (("rgb", slice(0, 3)), ("albedo", slice(3, 6))):
        ok, st = oracle.parity(g[:, sl], o[..., sl], kappa, tol)
        print(f"{label} {name}: max {st['max_rel']:.2e} (well-conditioned {st['max_rel_well_conditioned']:.2e}), "
              f"ill-conditioned {st['ill_conditioned']}/{st['n']}")
        assert ok, (label, name, st)


def _eval_both(mat, q, flags=0):
    dq = to_device(q)
    rgb, alb = mat.eval_albedo(dq, flags=flags)
    plain = mat.eval(dq, flags=flags).cpu().numpy()
    got = np.concatenate([rgb.cpu().numpy(), alb.cpu().numpy()], axis=1)
    assert np.array_equal(got[:, :3], plain)   # the RGB is nam_eval's
    return got


@pytest.mark.parametrize("cos", [False, True])
@pytest.mark.parametrize("H,NH,frame", [(64, 2, "mlp"), (16, 2, "none"), (64, 3, "paper")])
def test_albedo_fp32(gctx, oracle, cos, H, NH, frame):
    from paper_2305_02678_gb300 import binding as B
    W0, L, pyr, model, q = _setup(301 + H + NH, H=H, NH=NH, frame=frame, latent=np.float32)
    mat = gctx.material(W0, W0, L, pyr, model["frame"], model["decoder"], precision=B.NAM_PREC_F32)
    got = _eval_both(mat, q, B.NAM_OUT_COSINE if cos else 0)
    om = oracle.Model(W0, W0, L, pyr, model["frame"], model["decoder"], out_cosine=cos)
    _parity(oracle, got, oracle.eval(om, q), oracle.frame_condition(om, q), TOL_F32, f"fp32 {NH}x{H} {frame}")
    mat.destroy()
    gctx.check()


@pytest.mark.parametrize("H,NH,frame", [(64, 2, "mlp"), (32, 2, "none"), (64, 3, "paper")])
def test_albedo_fp16(gctx, oracle, H, NH, frame):
    from paper_2305_02678_gb300 import binding as B
    W0, L, pyr, model, q = _setup(311 + H + NH, H=H, NH=NH, frame=frame)
    mat = gctx.material(W0, W0, L, pyr, model["frame"], model["decoder"], precision=B.NAM_PREC_F16)
    got = _eval_both(mat, q, B.NAM_OUT_COSINE)
    om = oracle.Model(W0, W0, L, pyr, model["frame"], model["decoder"], params="fp16", out_cosine=True)
    _parity(oracle, got, oracle.eval(om, q), oracle.frame_condition(om, q), TOL_F16, f"fp16 {NH}x{H} {frame}")
    mat.destroy()
    gctx.check()


def test_albedo_fp8(gctx, oracle):
    from paper_2305_02678_gb300 import binding as B
    W0, L, pyr, model, q = _setup(321)
    om0 = oracle.Model(W0, W0, L, pyr, model["frame"], model["decoder"])
    amax = oracle.decoder_input_absmax(om0, q)
    scales = np.where(amax > 0, amax / 448.0, 1.0).astype(np.float32)
    mat = gctx.material(W0, W0, L, pyr, model["frame"], model["decoder"], precision=B.NAM_PREC_FP8, act_scale=scales)
    got = _eval_both(mat, q)
    om = oracle.Model(W0, W0, L, pyr, model["frame"], model["decoder"], params="fp8")
    _parity(oracle, got, oracle.eval(om, q), oracle.frame_condition(om, q), TOL_F8, "fp8")
    mat.destroy()
    gctx.check()


def test_albedo_multi_material_paths_give_rgb(gctx):
    """Binned and per-tile-selected evaluation of materials with the head
    give nam_eval's RGB (they write no albedo)."""
    import torch
    from paper_2305_02678_gb300 import binding as B
    mats = []
    for k in range(3):
        W0, L, pyr, model, q = _setup(331 + k, n=3000)
        mats.append(gctx.material(W0, W0, L, pyr, model["frame"], model["decoder"], precision=B.NAM_PREC_F16))
    dq = to_device(q)
    ids = np.repeat(np.arange(3, dtype=np.int32), 1000)
    tid = torch.from_numpy(ids).cuda()
    for fn in (B.nam_eval_binned, B.nam_eval_select):
        out = torch.full((3000, 3), -7.0, device="cuda")
        fn(gctx.h, [m.h for m in mats], dq, tid, 3000, out, torch.cuda.current_stream())
        got = out.cpu().numpy()
        for k, m in enumerate(mats):
            sel = np.nonzero(ids == k)[0]
            idx = torch.from_numpy(sel).cuda()
            ref = m.eval({f: t[idx].contiguous() for f, t in dq.items()}).cpu().numpy()
            assert np.array_equal(got[sel], ref)
    for m in mats:
        m.destroy()
    gctx.check()


def _train_setup(seed, n=3000, frame=True):
    rng = W.rng_streams(seed, 4)
    W0, L = 128, 8
    pyr = W.make_pyramid(rng[0], W0, W0, L, dtype=np.float32)
    model = W.make_model(rng[1], (14, 64, 64, 6), (8, 16, 6) if frame else None)
    q = W.uniform_queries(rng[2], n, 7.0)
    return W0, L, pyr, model, q, rng[3]


@pytest.mark.parametrize("frame", [True, False])
def test_albedo_backward(gctx, oracle, frame):
    import torch
    from paper_2305_02678_gb300 import binding as B
    W0, L, pyr, model, q, rng = _train_setup(341 + frame, frame=frame)
    om = oracle.Model(W0, W0, L, pyr, model["frame"], model["decoder"], out_cosine=True)
    keep = np.nonzero(oracle.frame_condition(om, q) <= 50.0)[0]
    q = {k: v[keep] for k, v in q.items()}
    n = len(keep)
    dl = rng.normal(0, 1, (n, 6)).astype(np.float32)
    mat = gctx.material(W0, W0, L, pyr, model["frame"], model["decoder"], precision=B.NAM_PREC_F32, trainable=True)
    gp = torch.zeros(mat.info.n_params, device="cuda")
    gz = torch.zeros((mat.info.texels, 8), device="cuda")
    B.nam_backward(gctx.h, mat.h, to_device(q), n, torch.from_numpy(dl).cuda(), gp, gz, torch.cuda.current_stream(),
                   B.NAM_OUT_COSINE)
    torch.cuda.synchronize()
    ref = oracle.grad(om, q, dl.astype(np.float64))
    for name, r, g in (("params", np.concatenate([ref["frame"], ref["decoder"]]), gp),
                       ("pyramid", ref["pyramid"].ravel(), gz.view(-1))):
        got = g.cpu().numpy().astype(np.float64)
        err = np.abs(got - r) / (np.abs(r) + 1e-2 * np.abs(r).max())
        print(f"frame={frame} {name}: max rel {err.max():.2e}")
        assert err.max() <= 1e-4
    mat.destroy()
    gctx.check()


def test_albedo_train_step_loss_and_direction(gctx, oracle):
    """The fused step's loss is the oracle's BRDF loss plus its albedo loss at
    the step's parameters; its first Adam update moves every parameter with
    a clear gradient against the sign of the oracle's gradient of that sum."""
    import torch
    from paper_2305_02678_gb300 import binding as B
    W0, L, pyr, model, q, rng = _train_setup(351, n=4096)
    target = W.ProceduralBRDF(rng)
    y = W.target_rgb(target, q)
    ya = W.albedo_targets(rng, target, q)
    mat = gctx.material(W0, W0, L, pyr, model["frame"], model["decoder"], precision=B.NAM_PREC_F32, trainable=True)
    p_dev, _ = mat.params()
    n_params = mat.info.n_params
    view = torch.as_tensor(_DevArray(p_dev, n_params), device="cuda")
    before = view.cpu().numpy().astype(np.float64)
    lr = 1e-4
    loss = B.nam_train_step_albedo(gctx.h, mat.h, to_device(q), torch.from_numpy(y).cuda(),
                                   torch.from_numpy(ya).cuda(), 4096, lr_params=lr, lr_pyramid=0.0, step=1,
                                   stream=torch.cuda.current_stream())
    after = view.cpu().numpy().astype(np.float64)
    om = oracle.Model(W0, W0, L, pyr, model["frame"], model["decoder"])
    o = oracle.eval(om, q)
    l_rgb, d_rgb = oracle.loss(o[:, :3], y)
    l_alb, d_alb = oracle.albedo_loss(o[:, 3:], ya)
    print(f"loss {loss:.6f}, oracle {l_rgb + l_alb:.6f} (BRDF {l_rgb:.6f} + albedo {l_alb:.6f})")
    assert abs(loss - (l_rgb + l_alb)) <= 1e-5 * (l_rgb + l_alb)
    g = oracle.grad(om, q, np.concatenate([d_rgb, d_alb], axis=1), with_pyramid=False)
    gref = np.concatenate([g["frame"], g["decoder"]])
    clear = np.abs(gref) > 1e-2 * np.abs(gref).max()
    step = after - before
    assert np.all(np.sign(step[clear]) == -np.sign(gref[clear]))
    assert np.allclose(np.abs(step[clear]), lr, rtol=1e-2)
    mat.destroy()
    gctx.check()


def _quadrature_albedo(target, u, v, wo, k=96):
    """Eq. 2 by a midpoint rule in (cos^2 theta, phi), where the
    cosine-weighted measure is uniform: integral = pi * mean f."""
    s = (np.arange(k) + 0.5) / k
    phi = (np.arange(k) + 0.5) / k * 2 * np.pi
    S, P = np.meshgrid(s, phi, indexing="ij")
    ct, st = np.sqrt(S.ravel()), np.sqrt(1 - S.ravel())
    wi = np.stack([st * np.cos(P.ravel()), st * np.sin(P.ravel()), ct])
    out = np.zeros((len(u), 3))
    for j in range(len(u)):
        m = wi.shape[1]
        f = target(np.full(m, u[j]), np.full(m, v[j]), wi, np.repeat(wo[:, j:j + 1], m, axis=1))
        out[j] = np.pi * f.mean(axis=0)
    return out


def test_albedo_head_learns_the_albedo(gctx):
    """300 steps of 8192 samples on the procedural material with one-sample
    albedo targets: the head's albedo at 64 test points (lod 0) approaches
    the quadrature of Eq. 2."""
    import torch
    from paper_2305_02678_gb300 import binding as B
    rng = W.rng_streams(361, 4)
    W0, L = 64, 7
    pyr = W.make_pyramid(rng[0], W0, W0, L, dtype=np.float32, std=0.1)
    model = W.make_model(rng[1], (14, 64, 64, 6), (8, 16, 6))
    target = W.ProceduralBRDF(rng[2])
    mat = gctx.material(W0, W0, L, pyr, model["frame"], model["decoder"], precision=B.NAM_PREC_F32, trainable=True)
    tq = W.uniform_queries(rng[3], 64, 0.0)
    wo = np.stack([tq["wox"], tq["woy"], tq["woz"]]).astype(np.float64)
    ref = _quadrature_albedo(target, tq["u"].astype(np.float64), tq["v"].astype(np.float64), wo)
    dtq = to_device(tq)

    def err():
        _, a = mat.eval_albedo(dtq)
        return float(np.mean(np.abs(a.cpu().numpy() - ref)))

    e0 = err()
    s = torch.cuda.current_stream()
    for step in range(1, 301):
        q = W.uniform_queries(rng[3], 8192, 0.0)
        y = torch.from_numpy(W.target_rgb(target, q)).cuda()
        ya = torch.from_numpy(W.albedo_targets(rng[3], target, q)).cuda()
        B.nam_train_step_albedo(gctx.h, mat.h, to_device(q), y, ya, 8192, lr_params=3e-3, lr_pyramid=1e-2,
                                step=step, stream=s, want_loss=False)
    e1 = err()
    print(f"mean |albedo - quadrature|: {e0:.4f} -> {e1:.4f} (reference mean {ref.mean():.3f})")
    assert e1 < 0.5 * e0 and e1 < 0.1
    mat.destroy()
    gctx.check()


def test_albedo_autograd(gctx, oracle):
    """NeuralMaterial with the head returns [n, 6]; autograd's gradient of
    sum(w * out) matches the oracle's reverse mode with dl = w."""
    import torch

    from paper_2305_02678_gb300.autograd import NeuralMaterial
    W0, L, pyr, model, q, rng = _train_setup(381, n=2000)
    om = oracle.Model(W0, W0, L, pyr, model["frame"], model["decoder"])
    keep = np.nonzero(oracle.frame_condition(om, q) <= 50.0)[0]
    q = {k: v[keep] for k, v in q.items()}
    n = len(keep)
    nm = NeuralMaterial(gctx, W0, W0, L, pyr, model["frame"], model["decoder"])
    out = nm(to_device(q))
    assert out.shape == (n, 6)
    w = torch.from_numpy(rng.normal(0, 1, (n, 6)).astype(np.float32)).cuda()
    (out * w).sum().backward()
    ref = oracle.grad(om, q, w.cpu().numpy().astype(np.float64), with_pyramid=False)
    r = np.concatenate([ref["frame"], ref["decoder"]])
    got = nm.params.grad.cpu().numpy().astype(np.float64)
    err = np.abs(got - r) / (np.abs(r) + 1e-2 * np.abs(r).max())
    print(f"autograd params: max rel {err.max():.2e}")
    assert err.max() <= 1e-4
    nm.material.destroy()
    gctx.check()


def test_albedo_refusals(gctx):
    import torch
    from paper_2305_02678_gb300 import binding as B
    W0, L, pyr, model, q, rng = _train_setup(371, n=256)
    alb = gctx.material(W0, W0, L, pyr, model["frame"], model["decoder"], precision=B.NAM_PREC_F32, trainable=True)
    m3 = W.make_model(rng, (14, 64, 64, 3), (8, 16, 6))
    rgb = gctx.material(W0, W0, L, pyr, m3["frame"], m3["decoder"], precision=B.NAM_PREC_F32, trainable=True)
    dq = to_device(q)
    y = torch.zeros((256, 3), device="cuda")
    with pytest.raises(B.NamError) as e:
        B.nam_train_step(gctx.h, alb.h, dq, y, 256, stream=torch.cuda.current_stream())
    assert e.value.status == B.NAM_ERR_UNSUPPORTED
    with pytest.raises(B.NamError) as e:
        B.nam_train_step_albedo(gctx.h, rgb.h, dq, y, y, 256, stream=torch.cuda.current_stream())
    assert e.value.status == B.NAM_ERR_UNSUPPORTED
    with pytest.raises(B.NamError) as e:
        B.nam_eval_albedo(gctx.h, rgb.h, dq, 256, y, y, torch.cuda.current_stream())
    assert e.value.status == B.NAM_ERR_UNSUPPORTED
    with pytest.raises(B.NamError) as e:
        gctx.material(W0, W0, L, pyr, model["frame"], model["decoder"], precision=B.NAM_PREC_F32, trainable=True,
                      encoder=W.make_mlp(rng, (4, 32, 32, 8)))
    assert e.value.status == B.NAM_ERR_UNSUPPORTED
    alb.destroy()
    rgb.destroy()
    gctx.check()


class _DevArray:
    """Zero-copy view of a libnam device buffer for torch (CUDA array interface)."""

    def __init__(self, ptr, n):
        self.__cuda_array_interface__ = {"shape": (n,), "typestr": "<f4", "data": (ptr, False), "version": 3}
