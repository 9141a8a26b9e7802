"""Pins of the oracle's encoder phase (Sec. 5.1: an MLP maps the material
parameters k(x) to the latent z(x), which goes to the decoder directly,
bypassing the latent texture): the encoder against a closed form and central
differences, the latent-input path against the texture path at texel centres
(where the filter returns one texel exactly), and dL/dz against the pyramid
gradient and central differences."""
import numpy as np
import pytest

import workloads as W


def _encoder(rng, widths):
    return [(rng.normal(0, 1.0 / np.sqrt(a), (b, a)), rng.normal(0, 0.1, b)) for a, b in zip(widths[:-1], widths[1:])]


def test_encoder_closed_form(oracle):
    """ReLU(k) - ReLU(-k) = k: W1 = [I; -I], W2 = I, W3 = [A, -A] give z = A k + c."""
    rng = np.random.default_rng(1)
    K = 4
    A = rng.normal(size=(8, K))
    c = rng.normal(size=8)
    W1 = np.concatenate([np.eye(K), -np.eye(K)])
    layers = [(W1, np.zeros(2 * K)), (np.eye(2 * K), np.zeros(2 * K)), (np.concatenate([A, -A], 1), c)]
    k = rng.normal(size=(50, K))
    assert np.allclose(oracle.encoder_forward(layers, k), k @ A.T + c, rtol=0, atol=1e-13)


def test_encoder_gradient_central_differences(oracle):
    rng = np.random.default_rng(2)
    layers = _encoder(rng, (4, 6, 6, 8))
    k = rng.normal(size=(30, 4))
    dz = rng.normal(size=(30, 8))
    g = oracle.encoder_grad(layers, k, dz)
    h = 1e-6
    checked = 0
    for l, (Wl, bl) in enumerate(layers):
        for arr, garr in ((Wl, g[l][0]), (bl, g[l][1])):
            for idx in list(np.ndindex(arr.shape))[::3]:
                old = arr[idx]
                arr[idx] = old + h
                fp = np.sum(dz * oracle.encoder_forward(layers, k))
                arr[idx] = old - h
                fm = np.sum(dz * oracle.encoder_forward(layers, k))
                arr[idx] = old
                fd = (fp - fm) / (2 * h)
                assert abs(fd - garr[idx]) <= 1e-6 * max(1.0, abs(fd)), (l, idx, fd, garr[idx])
                checked += 1
    assert checked > 30


def _texel_centre_setup(rng, n_side=8, frame=True, H=32):
    W0 = H0 = n_side
    pyr = W.make_pyramid(rng, W0, H0, 1, dtype=np.float32)
    model = W.make_model(rng, (14, H, H, 3), (8, 16, 6) if frame else None)
    xs, ys = np.meshgrid(np.arange(W0), np.arange(H0))
    xs, ys = xs.ravel(), ys.ravel()
    n = xs.size
    wi = rng.normal(size=(n, 3))
    wi[:, 2] = np.abs(wi[:, 2]) + 0.2
    wi /= np.linalg.norm(wi, axis=1, keepdims=True)
    wo = rng.normal(size=(n, 3))
    wo[:, 2] = np.abs(wo[:, 2]) + 0.2
    wo /= np.linalg.norm(wo, axis=1, keepdims=True)
    q = dict(u=((xs + 0.5) / W0).astype(np.float32), v=((ys + 0.5) / H0).astype(np.float32),
             lod=np.zeros(n, np.float32), wix=wi[:, 0].astype(np.float32), wiy=wi[:, 1].astype(np.float32),
             wiz=wi[:, 2].astype(np.float32), wox=wo[:, 0].astype(np.float32), woy=wo[:, 1].astype(np.float32),
             woz=wo[:, 2].astype(np.float32))
    texel = ys * W0 + xs
    return W0, H0, pyr, model, q, texel


@pytest.mark.parametrize("frame", [True, False])
def test_latent_input_matches_texture_at_texel_centres(oracle, frame):
    rng = np.random.default_rng(3)
    W0, H0, pyr, model, q, texel = _texel_centre_setup(rng, frame=frame)
    om = oracle.Model(W0, H0, 1, pyr, model["frame"], model["decoder"], out_cosine=True)
    y_tex = oracle.eval(om, q)
    qz = dict(q, z=pyr.astype(np.float64)[texel])
    y_z = oracle.eval(om, qz)
    assert np.array_equal(y_tex, y_z)
    dl = rng.normal(size=(len(texel), 3))
    g_tex = oracle.grad(om, q, dl)
    g_z = oracle.grad(om, qz, dl, with_z=True)
    assert np.allclose(g_tex["decoder"], g_z["decoder"], rtol=1e-12, atol=1e-14)
    assert np.allclose(g_tex["frame"], g_z["frame"], rtol=1e-12, atol=1e-14)
    # one query per texel, tap weight 1: dL/dz is that texel's gradient
    assert np.allclose(g_z["z"], g_tex["pyramid"][texel], rtol=1e-12, atol=1e-14)
    assert not np.any(g_z["pyramid"])


def test_latent_gradient_central_differences(oracle):
    rng = np.random.default_rng(4)
    W0, H0, pyr, model, q, texel = _texel_centre_setup(rng, n_side=4)
    om = oracle.Model(W0, H0, 1, pyr, model["frame"], model["decoder"])
    z = rng.normal(0, 0.5, (len(texel), 8))
    dl = rng.normal(size=(len(texel), 3))
    gz = oracle.grad(om, dict(q, z=z), dl, with_z=True)["z"]
    pat0 = oracle.relu_pattern(om, dict(q, z=z))
    h = 1e-6
    checked = 0
    for i in range(len(texel)):
        for c in range(8):
            zp, zm = z.copy(), z.copy()
            zp[i, c] += h
            zm[i, c] -= h
            if not (np.array_equal(oracle.relu_pattern(om, dict(q, z=zp)), pat0)
                    and np.array_equal(oracle.relu_pattern(om, dict(q, z=zm)), pat0)):
                continue
            fd = (np.sum(dl * oracle.eval(om, dict(q, z=zp))) - np.sum(dl * oracle.eval(om, dict(q, z=zm)))) / (2 * h)
            assert abs(fd - gz[i, c]) <= 1e-6 * max(1.0, abs(fd)), (i, c, fd, gz[i, c])
            checked += 1
    assert checked >= 100
