"""The encoder phase of training on the GPU (Sec. 5.1): nam_encode,
nam_backward_encoded and nam_encoder_bake against the oracle's FP64 encoder
and reverse mode, and the two-phase fit (encoder steps, bake, texel
finetuning) on the procedural material."""
import numpy as np
import pytest

import workloads as W
from conftest import to_device

pytestmark = pytest.mark.gpu

K = 4  # albedo RGB + roughness of the procedural material


def _setup(seed, n=4096, H=64, frame=True, W0=64, L=7):
    rng = W.rng_streams(seed, 5)
    pyr = W.make_pyramid(rng[0], W0, W0, L, dtype=np.float32)
    model = W.make_model(rng[1], (14, H, H, 3), (8, 16, 6) if frame else None)
    enc = W.make_mlp(rng[2], (K, 32, 32, 8))
    target = W.ProceduralBRDF(rng[3])
    q = W.uniform_queries(rng[4], n, float(L - 1))
    attrs = W.material_attributes(target, q)
    return W0, L, pyr, model, enc, target, q, attrs


def _rel(got, ref, floor):
    return np.abs(got - ref) / (np.abs(ref) + floor)


def _enc_err(oracle, enc, k, got):
    """|got - E(k)| over the magnitude of the terms that produce each output
    (the encoder run on |W|, |b|, |k|): the scale of FP32 rounding, which
    cancellation in a dot product does not shrink."""
    k = k.astype(np.float64)
    ref = oracle.encoder_forward(enc, k)
    mag = oracle.encoder_forward([(np.abs(Wl), np.abs(bl)) for Wl, bl in enc], np.abs(k))
    return np.abs(got.astype(np.float64) - ref) / mag


@pytest.mark.parametrize("n", [1, 127, 5000])
def test_encode_matches_oracle(gctx, oracle, n):
    import torch
    from paper_2305_02678_gb300 import binding as B
    W0, L, pyr, model, enc, target, q, attrs = _setup(31, n=max(n, 1))
    _encode_case(gctx, oracle, W0, L, pyr, model, enc, attrs, n)


@pytest.mark.parametrize("k_inputs", [1, 16])
def test_encode_input_widths(gctx, oracle, k_inputs):
    """The smallest and largest encoder input counts, on random parameters."""
    W0, L, pyr, model, _, _, _, _ = _setup(33)
    rng = np.random.default_rng(34 + k_inputs)
    enc = W.make_mlp(W.rng_streams(35 + k_inputs, 1)[0], (k_inputs, 32, 32, 8))
    attrs = rng.random((3001, k_inputs)).astype(np.float32)
    _encode_case(gctx, oracle, W0, L, pyr, model, enc, attrs, 3001)


def _encode_case(gctx, oracle, W0, L, pyr, model, enc, attrs, n):
    import torch
    from paper_2305_02678_gb300 import binding as B
    mat = gctx.material(W0, W0, L, pyr, model["frame"], model["decoder"], precision=B.NAM_PREC_F32,
                        trainable=True, encoder=enc)
    z = torch.empty((n, 8), device="cuda")
    B.nam_encode(gctx.h, mat.h, torch.from_numpy(attrs[:n]).cuda(), n, z, torch.cuda.current_stream())
    torch.cuda.synchronize()
    err = _enc_err(oracle, enc, attrs[:n], z.cpu().numpy())
    print(f"encode n={n}: max |err| / magnitude {err.max():.2e}")
    assert err.max() <= 1e-5
    mat.destroy()
    gctx.check()


@pytest.mark.parametrize("frame", [True, False])
@pytest.mark.parametrize("H", [32, 64])
def test_backward_encoded_matches_oracle(gctx, oracle, frame, H):
    import torch
    from paper_2305_02678_gb300 import binding as B
    W0, L, pyr, model, enc, target, q, attrs = _setup(41 + H, n=3000, H=H, frame=frame)
    om = oracle.Model(W0, W0, L, pyr, model["frame"], model["decoder"], out_cosine=True)
    z64 = oracle.encoder_forward(enc, attrs.astype(np.float64))
    keep = np.nonzero(oracle.frame_condition(om, dict(q, z=z64)) <= 50.0)[0]
    q = {k: v[keep] for k, v in q.items()}
    attrs, z64 = attrs[keep], z64[keep]
    n = len(keep)
    dl = np.random.default_rng(7).normal(0, 1, (n, 3)).astype(np.float32)
    mat = gctx.material(W0, W0, L, pyr, model["frame"], model["decoder"], precision=B.NAM_PREC_F32,
                        trainable=True, encoder=enc)
    gp = torch.zeros(mat.info.n_params, device="cuda")
    ge = torch.zeros(B.encoder_param_count(K), device="cuda")
    qd = {k: v for k, v in to_device(q).items() if k not in ("u", "v", "lod", "xi")}  # not read
    B.nam_backward_encoded(gctx.h, mat.h, qd, torch.from_numpy(attrs).cuda(), n, torch.from_numpy(dl).cuda(), gp, ge,
                           torch.cuda.current_stream(), B.NAM_OUT_COSINE)
    torch.cuda.synchronize()
    g = oracle.grad(om, dict(q, z=z64), dl.astype(np.float64), with_pyramid=False, with_z=True)
    ref_p = np.concatenate([g["frame"], g["decoder"]])
    got_p = gp.cpu().numpy().astype(np.float64)
    err_p = _rel(got_p, ref_p, 1e-2 * np.abs(ref_p).max())
    ref_e = oracle.flat_encoder(oracle.encoder_grad(enc, attrs.astype(np.float64), g["z"]))
    got_e = ge.cpu().numpy().astype(np.float64)
    err_e = _rel(got_e, ref_e, 1e-2 * np.abs(ref_e).max())
    print(f"H={H} frame={frame}: params max rel {err_p.max():.2e}, encoder max rel {err_e.max():.2e}")
    assert err_p.max() <= 1e-4 and err_e.max() <= 1e-4
    mat.destroy()
    gctx.check()


def test_encoder_bake_matches_oracle(gctx, oracle):
    import torch
    from paper_2305_02678_gb300 import binding as B
    W0, L, pyr, model, enc, target, q, attrs = _setup(51, n=16)
    mat = gctx.material(W0, W0, L, pyr, model["frame"], model["decoder"], precision=B.NAM_PREC_F32,
                        trainable=True, encoder=enc)
    ta = W.texel_attributes(target, W0, W0, L)
    B.nam_encoder_bake(gctx.h, mat.h, torch.from_numpy(ta).cuda(), torch.cuda.current_stream())
    torch.cuda.synchronize()
    _, pz = mat.params()
    texels = mat.info.texels
    got = torch.as_tensor(_DevArray(pz, texels * 8), device="cuda").view(texels, 8).cpu().numpy().astype(np.float64)
    err = _enc_err(oracle, enc, ta, got)
    print(f"bake: {texels} texels, max |err| / magnitude {err.max():.2e}")
    assert err.max() <= 1e-5
    mat.destroy()
    gctx.check()


def test_two_phase_fit(gctx):
    """Encoder phase, bake, then texel finetuning on the procedural target:
    the encoder phase lowers the loss, the baked texture starts the
    finetuning near where the encoder left off, and finetuning lowers it
    further."""
    import torch
    from paper_2305_02678_gb300 import binding as B
    W0, L, pyr, model, enc, target, q0, _ = _setup(61, n=16, W0=64, L=7)
    mat = gctx.material(W0, W0, L, pyr * 0.0, model["frame"], model["decoder"], precision=B.NAM_PREC_F32,
                        trainable=True, encoder=enc)
    rng = W.rng_streams(62, 1)[0]
    s = torch.cuda.current_stream()
    enc_losses = []
    for step in range(1, 201):
        q = W.uniform_queries(rng, 8192, 0.0)
        y = torch.from_numpy(W.target_rgb(target, q)).cuda()
        a = torch.from_numpy(W.material_attributes(target, q)).cuda()
        enc_losses.append(B.nam_train_step_encoded(gctx.h, mat.h, to_device(q), a, y, 8192, lr_params=3e-3,
                                                   step=step, stream=s))
    B.nam_encoder_bake(gctx.h, mat.h, torch.from_numpy(W.texel_attributes(target, W0, W0, L)).cuda(), s)
    fine = []
    for step in range(1, 101):
        q = W.uniform_queries(rng, 8192, 0.0)
        y = torch.from_numpy(W.target_rgb(target, q)).cuda()
        fine.append(B.nam_train_step(gctx.h, mat.h, to_device(q), y, 8192, lr_params=1e-3, lr_pyramid=1e-2,
                                     step=step, stream=s))
    e0, e1 = np.mean(enc_losses[:10]), np.mean(enc_losses[-10:])
    f0, f1 = np.mean(fine[:5]), np.mean(fine[-10:])
    print(f"encoder phase {e0:.4f} -> {e1:.4f}; finetuning {f0:.4f} -> {f1:.4f}")
    assert np.all(np.isfinite(enc_losses)) and np.all(np.isfinite(fine))
    assert e1 < 0.7 * e0
    assert f0 < 1.5 * e1
    assert f1 < f0
    mat.destroy()
    gctx.check()


class _DevArray:
    """Zero-copy view of a libnam device buffer for torch (CUDA array interface)."""

    def __init__(self, ptr, n):
        self.__cuda_array_interface__ = {"shape": (n,), "typestr": "<f4", "data": (ptr, False), "version": 3}
