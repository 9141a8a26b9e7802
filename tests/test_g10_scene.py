"""The synthetic-scene harness on the GPU against its FP64 version
(oracle/scene.py): the G-buffer of a ground plane and three spheres, and the
direct-lighting image rendered through nam_sample, nam_sample_pdf and
nam_eval on material-binned ranges."""
import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu

SCENE = {"width": 160, "height": 120, "eye": (0.0, 1.6, -6.0), "target": (0.0, 0.7, 0.0), "up": (0.0, 1.0, 0.0),
         "fov_y": 0.9, "ground_material": 0, "ground_y": 0.0, "ground_uv_scale": 2.0,
         "spheres": [(-1.6, 1.0, 0.0, 1.0, 1), (0.4, 0.6, -0.6, 0.6, 2), (1.9, 1.2, 1.0, 1.2, 3)],
         "sky_radiance": 1.5}


def _c_scene(B, sc):
    return B.make_scene(sc["width"], sc["height"], sc["eye"], sc["target"], sc["up"], sc["fov_y"], sc["spheres"],
                        sc["ground_y"], sc["ground_material"], sc["ground_uv_scale"], sc["sky_radiance"])


def test_gbuffer_matches_oracle(gctx):
    import torch

    import oracle.scene as S
    from paper_2305_02678_gb300 import binding as B
    n = SCENE["width"] * SCENE["height"]
    out = {"material": torch.empty(n, dtype=torch.int32, device="cuda")}
    for k, w in (("t", 1), ("u", 1), ("v", 1), ("lod", 1), ("frame", 9), ("view", 3)):
        out[k] = torch.empty((n, w) if w > 1 else n, device="cuda")
    B.nam_scene_gbuffer(gctx.h, _c_scene(B, SCENE), 256, out, torch.cuda.current_stream())
    torch.cuda.synchronize()
    ref = S.gbuffer(SCENE, 256)
    mat = out["material"].cpu().numpy()
    same = mat == ref["material"]
    print(f"material ids equal on {same.mean():.5f} of the pixels")
    assert same.mean() >= 0.999
    hit = same & (mat >= 0)
    g = {k: v.cpu().numpy().astype(np.float64) for k, v in out.items() if k != "material"}

    def check(name, err, tight, loose):
        err = err.reshape(len(err), -1).max(axis=1)
        print(f"{name}: 99th pct {np.percentile(err, 99):.1e}, max {err.max():.1e}")
        # FP32 ray casting: hits near a silhouette or at grazing angles on the
        # ground are ill-conditioned (the quadratic's discriminant, a small
        # direction component); the 99th percentile bounds the rest
        assert np.percentile(err, 99) <= tight and err.max() <= loose, name

    check("t", np.abs(g["t"][hit] - ref["t"][hit]) / ref["t"][hit], 1e-5, 1e-3)
    # uv in units of the pixel's filter footprint (2^lod level-0 texels)
    fp = np.exp2(ref["lod"][hit]) / 256
    du = np.abs(g["u"][hit] - ref["u"][hit])
    check("u", np.minimum(du, 1.0 - du) / fp, 1e-3, 5e-2)           # u wraps at the sphere's seam
    check("v", np.abs(g["v"][hit] - ref["v"][hit]) / fp, 1e-3, 5e-2)
    check("lod", np.abs(g["lod"][hit] - ref["lod"][hit]), 1e-4, 1e-2)
    # unit vectors from the FP32 hit point: errors of |t d| / r on a sphere
    check("frame", np.abs(g["frame"][hit] - ref["frame"][hit].reshape(-1, 9)), 1e-4, 2e-3)
    check("view", np.abs(g["view"][hit] - ref["view"][hit]), 1e-4, 2e-3)
    assert np.all(np.isinf(g["t"][mat < 0]))
    gctx.check()


def test_direct_lighting_matches_oracle(gctx, oracle):
    import torch

    import oracle.scene as S
    from paper_2305_02678_gb300 import binding as B
    rng = W.rng_streams(91, 10)
    W0, L = 256, 9
    mats, models, samplers = [], [], []
    for k in range(4):
        pyr = W.make_pyramid(rng[k], W0, W0, L, dtype=np.float16)
        model = W.make_model(rng[4 + k], (14, 64, 64, 3), (8, 16, 6))
        smp = W.make_mlp(rng[8], (11, 32, 32, 32, 9)) if k == 0 else W.make_mlp(W.rng_streams(92 + k, 1)[0],
                                                                               (11, 32, 32, 32, 9))
        mats.append(gctx.material(W0, W0, L, pyr, model["frame"], model["decoder"], precision=B.NAM_PREC_F16,
                                  sampler=smp))
        models.append(oracle.Model(W0, W0, L, pyr, model["frame"], model["decoder"], params="fp16",
                                   out_cosine=True))
        samplers.append(smp)
    n = SCENE["width"] * SCENE["height"]
    var = rng[9].random((n, 5)).astype(np.float32)
    img = torch.empty((n, 3), device="cuda")
    B.nam_scene_render_direct(gctx.h, _c_scene(B, SCENE), [m.h for m in mats], torch.from_numpy(var).cuda(), img,
                              torch.cuda.current_stream())
    torch.cuda.synchronize()
    got = img.cpu().numpy().astype(np.float64)
    ref = S.render_direct(SCENE, models, samplers, var.astype(np.float64), W0)
    sky = np.all(ref == SCENE["sky_radiance"], axis=1)
    assert np.all(got[sky] == SCENE["sky_radiance"])
    scale = np.abs(ref).mean()
    rel = np.abs(got - ref).max(axis=1) / (np.abs(ref).max(axis=1) + 1e-3 * scale)
    print(f"pixels: {n}, max rel {rel.max():.2e}, 99th pct {np.percentile(rel, 99):.2e}, "
          f"median {np.median(rel):.2e}; mean |diff| / mean |ref| {np.abs(got - ref).mean() / scale:.2e}")
    # FP16 evaluation on both sides; the sampled directions differ by FP32
    # rounding, which moves a rare shadow ray across a silhouette
    assert np.percentile(rel, 99) <= 2e-2
    assert np.abs(got - ref).mean() / scale <= 5e-3
    for m in mats:
        m.destroy()
    gctx.check()


def test_paths_match_oracle(gctx, oracle):
    """Three-vertex paths: the GPU harness against the FP64 version with the
    same variates.  Sampled directions differ by FP32 rounding, so a few
    paths take another turn at a silhouette; the bulk agrees closely."""
    import torch

    import oracle.scene as S
    from paper_2305_02678_gb300 import binding as B
    rng = W.rng_streams(95, 10)
    W0, L = 256, 9
    sc = dict(SCENE, width=96, height=72)
    mats, models, samplers = [], [], []
    for k in range(4):
        pyr = W.make_pyramid(rng[k], W0, W0, L, dtype=np.float16)
        model = W.make_model(rng[4 + k], (14, 64, 64, 3), (8, 16, 6))
        smp = W.make_mlp(W.rng_streams(96 + k, 1)[0], (11, 32, 32, 32, 9))
        mats.append(gctx.material(W0, W0, L, pyr, model["frame"], model["decoder"], precision=B.NAM_PREC_F16,
                                  sampler=smp))
        models.append(oracle.Model(W0, W0, L, pyr, model["frame"], model["decoder"], params="fp16",
                                   out_cosine=True))
        samplers.append(smp)
    n = sc["width"] * sc["height"]
    bounces = 3
    var = rng[9].random((bounces, n, 5)).astype(np.float32)
    img = torch.empty((n, 3), device="cuda")
    B.nam_scene_render_paths(gctx.h, _c_scene(B, sc), [m.h for m in mats], bounces, torch.from_numpy(var).cuda(),
                             img, torch.cuda.current_stream())
    torch.cuda.synchronize()
    got = img.cpu().numpy().astype(np.float64)
    ref = S.render_paths(sc, models, samplers, var.astype(np.float64), W0, bounces)
    direct = S.render_direct(sc, models, samplers, var[0].astype(np.float64), W0)
    scale = np.abs(ref).mean()
    rel = np.abs(got - ref).max(axis=1) / (np.abs(ref).max(axis=1) + 1e-3 * scale)
    print(f"paths: median rel {np.median(rel):.2e}, 95th pct {np.percentile(rel, 95):.2e}, max {rel.max():.2e}; "
          f"mean |diff| / mean |ref| {np.abs(got - ref).mean() / scale:.2e}; "
          f"indirect share {np.abs(ref - direct).mean() / scale:.2f}")
    # the harness evaluates the FP16 weights with FP64 activations; the GPU's
    # FP16 evaluations differ from that by ~3e-4 on average, which bounds the
    # median path here
    assert np.median(rel) <= 5e-4
    assert np.percentile(rel, 95) <= 2e-2
    assert np.abs(got - ref).mean() / scale <= 1e-2
    # later vertices contribute (random decoders can return negative values,
    # so the indirect term is not a sum of positive parts)
    assert np.abs(ref - direct).mean() > 0.01 * scale
    for m in mats:
        m.destroy()
    gctx.check()


def test_paths_one_vertex_is_direct_and_arguments(gctx):
    import torch
    from paper_2305_02678_gb300 import binding as B
    rng = W.rng_streams(97, 9)
    mats = []
    for k in range(4):
        pyr = W.make_pyramid(rng[k], 64, 64, 7, dtype=np.float16)
        model = W.make_model(rng[4 + k], (14, 64, 64, 3), (8, 16, 6))
        mats.append(gctx.material(64, 64, 7, pyr, model["frame"], model["decoder"], precision=B.NAM_PREC_F16,
                                  sampler=W.make_mlp(W.rng_streams(98 + k, 1)[0], (11, 32, 32, 32, 9))))
    sc = dict(SCENE, width=64, height=48)
    n = 64 * 48
    var = torch.from_numpy(rng[8].random((1, n, 5)).astype(np.float32)).cuda()
    a = torch.empty((n, 3), device="cuda")
    b = torch.empty((n, 3), device="cuda")
    h = [m.h for m in mats]
    B.nam_scene_render_direct(gctx.h, _c_scene(B, sc), h, var[0], a)
    B.nam_scene_render_paths(gctx.h, _c_scene(B, sc), h, 1, var, b)
    torch.cuda.synchronize()
    assert torch.equal(a, b)
    for bad in (0, B.NAM_SCENE_MAX_BOUNCES + 1):
        with pytest.raises(B.NamError) as e:
            B.nam_scene_render_paths(gctx.h, _c_scene(B, sc), h, bad, var, b)
        assert e.value.status == B.NAM_ERR_INVALID_ARG
    with pytest.raises(B.NamError) as e:   # the scene names material 3; give three
        B.nam_scene_render_direct(gctx.h, _c_scene(B, sc), h[:3], var[0], a)
    assert e.value.status == B.NAM_ERR_INVALID_ARG
    for m in mats:
        m.destroy()
    gctx.check()
