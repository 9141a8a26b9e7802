"""Pins of the scene harness's FP64 version (oracle/scene.py): hits, uv,
frames and levels of detail at pixels worked out by hand, orthonormal
right-handed frames, and the direct-lighting estimator with a constant
material (reflected radiance pi c L in expectation)."""
import numpy as np
import pytest

import workloads as W


def _sphere_scene():
    return {"width": 3, "height": 3, "eye": (0.0, 1.0, -5.0), "target": (0.0, 1.0, 0.0), "up": (0.0, 1.0, 0.0),
            "fov_y": 0.5, "ground_material": -1, "ground_y": 0.0, "ground_uv_scale": 1.0,
            "spheres": [(0.0, 1.0, 0.0, 1.0, 0)], "sky_radiance": 1.0}


def test_sphere_hit_by_hand():
    import oracle.scene as S
    g = S.gbuffer(_sphere_scene(), 256)
    c = 4  # centre pixel of 3 x 3: the view axis
    assert g["material"][c] == 0
    assert np.isclose(g["t"][c], 4.0, rtol=1e-14)
    assert np.isclose(g["u"][c], 0.25, atol=1e-14) and np.isclose(g["v"][c], 0.5, atol=1e-14)
    assert np.allclose(g["frame"][c], [[1, 0, 0], [0, -1, 0], [0, 0, -1]], atol=1e-14)
    assert np.allclose(g["view"][c], [0, 0, 1], atol=1e-14)
    # ray cone: spread 2 tan(0.25) / 3 per unit, t = 4, normal incidence, s = 1 / (pi sqrt 2)
    fp = 2 * np.tan(0.25) / 3 * 4.0 / (np.pi * np.sqrt(2.0)) * 256
    assert np.isclose(g["lod"][c], np.log2(fp), rtol=1e-13)


def test_ground_hit_by_hand():
    import oracle.scene as S
    sc = {"width": 5, "height": 5, "eye": (0.3, 2.0, 0.2), "target": (0.3, 0.0, 0.2), "up": (0.0, 0.0, 1.0),
          "fov_y": 0.8, "ground_material": 2, "ground_y": 0.0, "ground_uv_scale": 4.0, "spheres": [],
          "sky_radiance": 1.0}
    g = S.gbuffer(sc, 1024)
    c = 12
    assert g["material"][c] == 2 and np.isclose(g["t"][c], 2.0, rtol=1e-14)
    assert np.isclose(g["u"][c], 0.3 / 4.0) and np.isclose(g["v"][c], 0.2 / 4.0)
    assert np.allclose(g["frame"][c], [[1, 0, 0], [0, 0, -1], [0, 1, 0]], atol=1e-14)
    assert np.isclose(g["lod"][c], np.log2(2 * np.tan(0.4) / 5 * 2.0 / 4.0 * 1024), rtol=1e-13)
    assert np.all(g["material"] == 2)  # every ray looks down at the plane


def test_frames_orthonormal_right_handed():
    import oracle.scene as S
    sc = {"width": 64, "height": 48, "eye": (0.0, 1.5, -6.0), "target": (0.0, 0.8, 0.0), "up": (0.0, 1.0, 0.0),
          "fov_y": 0.9, "ground_material": 0, "ground_y": 0.0, "ground_uv_scale": 2.0,
          "spheres": [(-1.2, 1.0, 0.0, 1.0, 1), (1.3, 0.7, 0.5, 0.7, 2)], "sky_radiance": 1.0}
    g = S.gbuffer(sc, 256)
    hit = g["material"] >= 0
    F = g["frame"][hit]
    assert np.allclose(np.einsum("nij,nkj->nik", F, F), np.eye(3)[None], atol=1e-12)
    assert np.allclose(np.linalg.det(F), 1.0, atol=1e-12)
    assert np.all(g["view"][hit][:, 2] > 0)  # every visible surface faces the eye
    assert set(np.unique(g["material"])) == {-1, 0, 1, 2}


def test_constant_material_direct_lighting(oracle):
    """Decoder with zero weights and output bias c: f cos = c cos, the
    reflected sky light is pi c L, and the MIS estimate (BSDF sample from the
    random sampler network plus cosine light sample) averages to it."""
    import oracle.scene as S
    rng = W.rng_streams(81, 4)
    pyr = W.make_pyramid(rng[0], 16, 16, 5, dtype=np.float32)
    H = 16
    c = np.array([0.2, 0.5, 0.8], np.float32)
    dec = [(np.zeros((H, 14), np.float32), np.zeros(H, np.float32)), (np.zeros((H, H), np.float32), np.zeros(H, np.float32)),
           (np.zeros((3, H), np.float32), c)]
    model = oracle.Model(16, 16, 5, pyr, None, dec, out_cosine=True)
    sampler = W.make_mlp(rng[1], (11, 32, 32, 32, 9))
    sc = {"width": 64, "height": 64, "eye": (0.0, 3.0, 0.0), "target": (0.0, 0.0, 0.01), "up": (0.0, 0.0, 1.0),
          "fov_y": 0.6, "ground_material": 0, "ground_y": 0.0, "ground_uv_scale": 3.0, "spheres": [],
          "sky_radiance": 2.0}
    var = rng[2].random((64 * 64, 5))
    img = S.render_direct(sc, [model], [sampler], var, 16)
    expect = np.pi * c * 2.0
    mean = img.mean(axis=0)
    sem = img.std(axis=0) / np.sqrt(len(img))
    assert np.all(np.abs(mean - expect) <= 4 * sem + 1e-12), (mean, expect, sem)
