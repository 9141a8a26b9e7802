"""The torch.autograd.Function over nam_eval / nam_backward: gradients equal
the oracle's reverse mode, a torch-side loss + torch.optim.Adam step equals
nam_train_step, and fitting the procedural GGX target through it lowers the
loss."""
import numpy as np
import pytest

import workloads as W
from conftest import to_device

pytestmark = pytest.mark.gpu


def _setup(seed, n=4096, frame=True):
    rng = W.rng_streams(seed, 4)
    W0 = H0 = 128
    L = 8
    pyr = W.make_pyramid(rng[0], W0, H0, L, dtype=np.float32)
    model = W.make_model(rng[1], (14, 64, 64, 3), (8, 16, 6) if frame else None)
    q = W.uniform_queries(rng[2], n, 7.0)
    dl = rng[3].normal(0, 1, (n, 3)).astype(np.float32)
    return W0, H0, L, pyr, model, q, dl


@pytest.mark.parametrize("frame", [True, False])
def test_autograd_gradient_matches_oracle(gctx, oracle, frame):
    import torch
    from paper_2305_02678_gb300.autograd import NeuralMaterial
    W0, H0, L, pyr, model, q, dl = _setup(71, frame=frame)
    om = oracle.Model(W0, H0, L, pyr, model["frame"], model["decoder"], out_cosine=True)
    k = oracle.frame_condition(om, q)
    keep = np.nonzero(k <= 50.0)[0]
    q = {f: v[keep] for f, v in q.items()}
    dl = dl[keep]
    nm = NeuralMaterial(gctx, W0, H0, L, pyr, model["frame"], model["decoder"])
    rgb = nm(to_device(q), cosine=True)
    ok, st = oracle.parity(rgb.detach().cpu().numpy(), oracle.eval(om, q), k[keep], 1e-5)
    assert ok, st
    (rgb * torch.from_numpy(dl).cuda()).sum().backward()
    ref = oracle.grad(om, q, dl.astype(np.float64))
    ref_params = np.concatenate([ref["frame"], ref["decoder"]])
    got = nm.params.grad.cpu().numpy().astype(np.float64)
    err = np.abs(got - ref_params) / (np.abs(ref_params) + 1e-2 * np.abs(ref_params).max())
    assert err.max() <= 1e-4, err.max()
    gz = nm.pyramid.grad.cpu().numpy().astype(np.float64)
    errz = np.abs(gz - ref["pyramid"]) / (np.abs(ref["pyramid"]) + 1e-2 * np.abs(ref["pyramid"]).max())
    assert errz.max() <= 1e-4, errz.max()
    nm.material.destroy()


def test_torch_adam_step_matches_library_train_step(gctx):
    """Two steps of (torch log-L1 loss, autograd backward, torch.optim.Adam)
    against two nam_train_step calls on an identical material."""
    import torch
    from paper_2305_02678_gb300 import binding as B
    from paper_2305_02678_gb300.autograd import NeuralMaterial, log_l1_loss, material_tensors
    rng = W.rng_streams(72, 4)
    W0 = H0 = 128
    L = 8
    pyr = W.make_pyramid(rng[0], W0, H0, L, dtype=np.float32)
    model = W.make_model(rng[1], (14, 64, 64, 3), (8, 16, 6))
    target = W.ProceduralBRDF(rng[2])
    nm = NeuralMaterial(gctx, W0, H0, L, pyr, model["frame"], model["decoder"])
    lib = gctx.material(W0, H0, L, pyr, model["frame"], model["decoder"], precision=B.NAM_PREC_F32, trainable=True)
    opt = torch.optim.Adam([{"params": [nm.params], "lr": 1e-3}, {"params": [nm.pyramid], "lr": 1e-2}],
                           betas=(0.9, 0.999), eps=1e-8)
    n = 16384
    for step in (1, 2):
        q = W.uniform_queries(rng[3], n, 7.0)
        y = torch.from_numpy(W.target_rgb(target, q)).cuda()
        dq = to_device(q)
        opt.zero_grad()
        loss = log_l1_loss(nm(dq), y)
        loss.backward()
        opt.step()
        l_lib = B.nam_train_step(gctx.h, lib.h, dq, y, n, lr_params=1e-3, lr_pyramid=1e-2, step=step,
                                 stream=torch.cuda.current_stream())
        assert abs(loss.item() - l_lib) <= 1e-5 * abs(l_lib), (loss.item(), l_lib)
    torch.cuda.synchronize()
    p_lib, z_lib = material_tensors(lib)
    # Adam's early updates are ~lr * sign(gradient) whatever the gradient's
    # size, so an entry whose summed gradient is ~0 (atomics add in a
    # different order in the two runs) may move by up to 2 lr per step in
    # opposite directions.  Everything else agrees to FP32 rounding.
    for got, ref, lr in ((nm.params.detach(), p_lib, 1e-3), (nm.pyramid.detach().ravel(), z_lib.ravel(), 1e-2)):
        d = (got - ref).abs()
        assert d.max().item() <= 4 * lr * 1.001
        frac = (d > 1e-6 + 1e-5 * ref.abs()).float().mean().item()
        assert frac <= 1e-3, frac
    lib.destroy()
    nm.material.destroy()
    gctx.check()


def test_fit_procedural_brdf_through_autograd(gctx):
    import torch
    from paper_2305_02678_gb300.autograd import NeuralMaterial, log_l1_loss
    w = W.workload(4, scale=1 / 16)
    m = w["model"]
    nm = NeuralMaterial(gctx, w["W0"], w["H0"], w["L"], w["pyramid"], m["frame"], m["decoder"])
    opt = torch.optim.Adam([{"params": [nm.params], "lr": 1e-3}, {"params": [nm.pyramid], "lr": 1e-2}])
    rng = W.rng_streams(73, 1)[0]
    losses = []
    for _ in range(120):
        q = W.uniform_queries(rng, 16384, 10.0)
        y = torch.from_numpy(W.target_rgb(w["target"], q)).cuda()
        opt.zero_grad()
        loss = log_l1_loss(nm(to_device(q)), y)
        loss.backward()
        opt.step()
        losses.append(loss.item())
    first, last = np.mean(losses[:10]), np.mean(losses[-10:])
    print(f"autograd fit: loss {first:.4f} -> {last:.4f}")
    assert np.all(np.isfinite(losses)) and last < 0.7 * first
    nm.material.destroy()


def test_autograd_rejects_foreign_tensors(gctx):
    import torch
    from paper_2305_02678_gb300.autograd import NeuralBRDFFunction, NeuralMaterial
    W0, H0, L, pyr, model, q, _ = _setup(74, n=256)
    nm = NeuralMaterial(gctx, W0, H0, L, pyr, model["frame"], model["decoder"])
    other = torch.zeros_like(nm.params, requires_grad=True)
    with pytest.raises(ValueError):
        NeuralBRDFFunction.apply(other, nm.pyramid, nm.material, to_device(q), 0)
    nm.material.destroy()
