"""Reverse mode on the GPU (nam_backward, nam_train_step) against the oracle's
gradient and against central differences of the GPU forward."""
import numpy as np
import pytest

import workloads as W
from conftest import to_device

pytestmark = pytest.mark.gpu


class _DevArray:
    """Zero-copy view of a libnam device buffer for torch (CUDA array interface)."""

    def __init__(self, ptr, n):
        self.__cuda_array_interface__ = {"shape": (n,), "typestr": "<f4", "data": (ptr, False), "version": 3}


def _small_train_setup(seed, n=4096, H=64, frame=True, filt=0):
    rng = W.rng_streams(seed, 4)
    W0 = H0 = 128
    L = 8
    pyr = W.make_pyramid(rng[0], W0, H0, L, dtype=np.float32)
    model = W.make_model(rng[1], (14, H, H, 3), (8, 16, 6) if frame else None)
    q = W.uniform_queries(rng[2], n, 7.0)
    dl = rng[3].normal(0, 1, (n, 3)).astype(np.float32)
    return W0, H0, L, pyr, model, q, dl


def _well_conditioned(oracle, om, q, limit=50.0):
    k = oracle.frame_condition(om, q)
    idx = np.nonzero(k <= limit)[0]
    return {f: v[idx] for f, v in q.items()}


@pytest.mark.parametrize("frame", [True, False])
@pytest.mark.parametrize("filt", [0, 1])
@pytest.mark.parametrize("H", [16, 32, 64])
def test_backward_matches_oracle_gradient(gctx, oracle, frame, filt, H):
    import torch
    from paper_2305_02678_gb300 import binding as B
    W0, H0, L, pyr, model, q, dl = _small_train_setup(11 + H + filt, H=H, frame=frame, filt=filt)
    om = oracle.Model(W0, H0, L, pyr, model["frame"], model["decoder"], filter=filt, out_cosine=True)
    q = _well_conditioned(oracle, om, q)
    n = len(q["u"])
    dl = dl[:n]
    mat = gctx.material(W0, H0, L, pyr, model["frame"], model["decoder"], precision=B.NAM_PREC_F32,
                        filter=filt, trainable=True)
    gp = torch.zeros(mat.info.n_params, device="cuda")
    gz = torch.zeros((mat.info.texels, 8), device="cuda")
    B.nam_backward(gctx.h, mat.h, to_device(q), n, torch.from_numpy(dl).cuda(), gp, gz,
                   torch.cuda.current_stream(), B.NAM_OUT_COSINE)
    torch.cuda.synchronize()
    ref = oracle.grad(om, q, dl.astype(np.float64))
    ref_params = np.concatenate([ref["frame"], ref["decoder"]])
    got = gp.cpu().numpy().astype(np.float64)
    # near-zero entries (sums over the batch that cancel) compare against 1%
    # of the largest gradient: FP32 accumulation order differs from FP64
    scale = np.abs(ref_params).max()
    err = np.abs(got - ref_params) / (np.abs(ref_params) + 1e-2 * scale)
    print(f"params H={H} frame={frame} filt={filt}: max rel {err.max():.2e}")
    assert err.max() <= 1e-4
    gzr = ref["pyramid"]
    gzg = gz.cpu().numpy().astype(np.float64)
    sc = np.abs(gzr).max()
    errz = np.abs(gzg - gzr) / (np.abs(gzr) + 1e-2 * sc)
    print(f"pyramid: max rel {errz.max():.2e}")
    assert errz.max() <= 1e-4
    mat.destroy()
    gctx.check()


def test_backward_accumulates_and_handles_ragged_batches(gctx):
    import torch
    from paper_2305_02678_gb300 import binding as B
    W0, H0, L, pyr, model, q, dl = _small_train_setup(21, n=1000)
    mat = gctx.material(W0, H0, L, pyr, model["frame"], model["decoder"], precision=B.NAM_PREC_F32, trainable=True)
    dq = to_device(q)
    dlt = torch.from_numpy(dl).cuda()
    g1 = torch.zeros(mat.info.n_params, device="cuda")
    B.nam_backward(gctx.h, mat.h, dq, 1000, dlt, g1, None, torch.cuda.current_stream())
    g2 = torch.zeros_like(g1)
    # same batch as a 129-query and an 871-query launch: gradients add up
    for s, c in ((0, 129), (129, 871)):
        sub = {k: v[s:s + c] for k, v in dq.items()}
        B.nam_backward(gctx.h, mat.h, sub, c, dlt[s:s + c], g2, None, torch.cuda.current_stream())
    torch.cuda.synchronize()
    assert torch.allclose(g1, g2, rtol=1e-5, atol=1e-6 * g1.abs().max().item())
    mat.destroy()


def test_gpu_gradient_against_central_differences(gctx, oracle):
    """Central differences (h = 1e-3) of the GPU FP32 forward, the sum
    <dl, y> reduced in FP64 on the GPU, on 64 random parameters."""
    import torch
    from paper_2305_02678_gb300 import binding as B
    W0, H0, L, pyr, model, q, dl = _small_train_setup(31, n=2048)
    om = oracle.Model(W0, H0, L, pyr, model["frame"], model["decoder"])
    q = _well_conditioned(oracle, om, q)
    n = len(q["u"])
    dl = dl[:n]
    mat = gctx.material(W0, H0, L, pyr, model["frame"], model["decoder"], precision=B.NAM_PREC_F32, trainable=True)
    pptr, zptr = mat.params()
    P = torch.as_tensor(_DevArray(pptr, mat.info.n_params), device="cuda")
    Z = torch.as_tensor(_DevArray(zptr, mat.info.texels * 8), device="cuda")
    dq = to_device(q)
    dlt = torch.from_numpy(dl).cuda()
    gp = torch.zeros(mat.info.n_params, device="cuda")
    gz = torch.zeros(mat.info.texels * 8, device="cuda")
    B.nam_backward(gctx.h, mat.h, dq, n, dlt, gp, gz, torch.cuda.current_stream())
    out = torch.empty((n, 3), device="cuda")
    pattern0 = oracle.relu_pattern(om, q)

    def J():
        B.nam_eval(gctx.h, mat.h, dq, n, out, torch.cuda.current_stream())
        return float((out.double() * dlt.double()).sum().item())

    rng = np.random.default_rng(5)
    h = 1e-3
    checked = redrawn = 0
    for buf, grad, count, kind in ((P, gp, mat.info.n_params, "param"), (Z, gz, mat.info.texels * 8, "texel")):
        want = 48 if kind == "param" else 16
        done = 0
        for i in rng.permutation(count):
            if done == want:
                break
            x0 = float(buf[i].item())
            if kind == "texel" and abs(float(grad[i].item())) == 0.0:
                continue
            vals = []
            kink = False
            for sgn in (1, -1):
                buf[i] = x0 + sgn * h
                step = abs(float(buf[i].item()) - x0)
                vals.append((J(), step))
                # the oracle decides whether the step crosses a ReLU kink
                fr = oracle.Model(W0, H0, L, pyr, model["frame"], model["decoder"])
                if kind == "param":
                    flat = P.cpu().numpy().astype(np.float64)
                    fr.frame_params[:] = flat[:fr.frame_params.size]
                    fr.dec_params[:] = flat[fr.frame_params.size:]
                else:
                    fr._pyr[...] = Z.cpu().numpy().reshape(-1, 8)
                kink |= not np.array_equal(oracle.relu_pattern(fr, q), pattern0)
            buf[i] = x0
            if kink:
                redrawn += 1
                continue
            fd = (vals[0][0] - vals[1][0]) / (vals[0][1] + vals[1][1])
            an = float(grad[i].item())
            # FP32 forward: |J| rounding ~ 1e-7 sum|dl y| per evaluation
            slack = 4e-7 * float((out.abs().double() * dlt.abs().double()).sum().item()) / h
            assert abs(fd - an) <= 2e-3 * abs(an) + slack, (kind, i, fd, an, slack)
            done += 1
            checked += 1
    assert checked == 64
    print(f"checked 64 parameters, {redrawn} re-drawn for kinks")
    mat.destroy()


def test_train_step_reduces_loss(gctx):
    """Fit the procedural GGX-over-Lambert target (Adam, log-space L1)."""
    import torch
    from paper_2305_02678_gb300 import binding as B
    w = W.workload(4, scale=1 / 16)
    m = w["model"]
    mat = gctx.material(w["W0"], w["H0"], w["L"], w["pyramid"], m["frame"], m["decoder"], precision=B.NAM_PREC_F32,
                        trainable=True)
    rng = W.rng_streams(40, 1)[0]
    losses = []
    for step in range(1, 121):
        q = W.uniform_queries(rng, 16384, 10.0)
        y = W.target_rgb(w["target"], q)
        loss = B.nam_train_step(gctx.h, mat.h, to_device(q), torch.from_numpy(y).cuda(), 16384, lr_params=1e-3,
                                lr_pyramid=1e-2, step=step, stream=torch.cuda.current_stream())
        losses.append(loss)
    first, last = np.mean(losses[:10]), np.mean(losses[-10:])
    print(f"loss {first:.4f} -> {last:.4f}")
    assert np.all(np.isfinite(losses))
    assert last < 0.7 * first
    mat.destroy()
    gctx.check()
