"""Pins of the oracle's albedo head (the paper's albedo inference: the
decoder outputs an extra RGB triplet, fitted with an L2 loss to one-sample
Monte Carlo estimates of the directional albedo of Eq. 2).  Each pin rests
on something other than the oracle's own formulas: a 6-output decoder split
into two 3-output decoders, the definition of the cosine factor, central
finite differences, a hand-computed loss, and a quadrature of Eq. 2 for the
training targets."""
import numpy as np
import pytest

import workloads as W

from test_oracle_pins import _flat_frame, _unflat_dec, _unflat_frame


def _setup(seed, n=256):
    rng = np.random.default_rng(seed)
    W0 = H0 = 16
    L = 5
    pyr = rng.normal(0, 0.5, (W.pyramid_texel_count(W0, H0, L), 8)).astype(np.float32)
    model = W.make_model(rng, (14, 32, 32, 6), (8, 16, 6))
    q = W.uniform_queries(rng, n, 4.0)
    return W0, H0, L, pyr, model, q, rng


def test_six_outputs_are_two_three_output_decoders(oracle):
    """Outputs 0..2 are the decoder with the first three output rows;
    outputs 3..5 the decoder with the last three, without the cosine factor.
    A swapped, transposed or shifted output row fails this."""
    W0, H0, L, pyr, model, q, _ = _setup(21)
    dec = model["decoder"]
    Wo, bo = dec[-1]
    rgb_dec = dec[:-1] + [(Wo[:3], bo[:3])]
    alb_dec = dec[:-1] + [(Wo[3:], bo[3:])]
    for cos in (False, True):
        y6 = oracle.eval(oracle.Model(W0, H0, L, pyr, model["frame"], dec, out_cosine=cos), q)
        assert y6.shape == (256, 6)
        rgb = oracle.eval(oracle.Model(W0, H0, L, pyr, model["frame"], rgb_dec, out_cosine=cos), q)
        alb = oracle.eval(oracle.Model(W0, H0, L, pyr, model["frame"], alb_dec, out_cosine=False), q)
        assert np.array_equal(y6[:, :3], rgb)
        assert np.array_equal(y6[:, 3:], alb)


def test_cosine_factor_on_rgb_only(oracle):
    """out_cosine multiplies the BRDF by max(0, wi.z) and leaves the albedo
    (a function of x and wo alone) as it is."""
    W0, H0, L, pyr, model, q, _ = _setup(22)
    q = dict(q)
    q["wiz"] = q["wiz"].copy()
    q["wiz"][::3] *= -1.0   # some wi below the horizon
    a = oracle.eval(oracle.Model(W0, H0, L, pyr, model["frame"], model["decoder"], out_cosine=False), q)
    b = oracle.eval(oracle.Model(W0, H0, L, pyr, model["frame"], model["decoder"], out_cosine=True), q)
    cz = np.maximum(q["wiz"].astype(np.float64), 0.0)
    assert np.array_equal(b[:, 3:], a[:, 3:])
    assert np.allclose(b[:, :3], a[:, :3] * cz[:, None], rtol=1e-15, atol=0.0)


def test_albedo_gradient_matches_central_differences(oracle):
    """Reverse mode of a 6-output decoder with out_cosine: 24 random decoder
    parameters (the output rows of both triplets among them), 8 frame
    parameters and 8 texels, against Richardson-extrapolated central
    differences of sum <dl, y> with dl [n, 6]."""
    W0, H0, L, pyr, model, q, rng = _setup(23)
    dl = rng.normal(0, 1, (256, 6))
    widths = (14, 32, 32, 6)
    fr0 = _flat_frame(model["frame"]).astype(np.float32)
    dec0 = np.concatenate([np.concatenate([Wt.ravel(), b]) for Wt, b in model["decoder"]]).astype(np.float32)

    def model_of(fr, dec, p):
        return oracle.Model(W0, H0, L, p, _unflat_frame(fr, 16), _unflat_dec(dec, widths), out_cosine=True)

    base = oracle.Model(W0, H0, L, pyr, model["frame"], model["decoder"], out_cosine=True)
    g = oracle.grad(base, q, dl)
    pattern0 = oracle.relu_pattern(base, q)
    arrs = {"frame": fr0, "decoder": dec0, "pyramid": pyr}
    # the output layer's parameters: rows 0..2 and 3..5 of Wo and bo
    n_out = 32 * 6 + 6
    out_idx = np.arange(dec0.size - n_out, dec0.size)
    picks = {"frame": rng.permutation(fr0.size),
             "decoder": np.concatenate([rng.permutation(out_idx)[:12], rng.permutation(dec0.size - n_out)]),
             "pyramid": rng.permutation(pyr.size)}
    want = {"frame": 8, "decoder": 24, "pyramid": 8}
    for kind in ("frame", "decoder", "pyramid"):
        done = 0
        n_out_done = 0
        for i in picks[kind]:
            if done == want[kind]:
                break
            x0 = float(arrs[kind].ravel()[i])
            kink = False
            fds = []
            for step in (1e-3, 5e-4):
                vals, steps = [], []
                for sgn in (+1, -1):
                    a = {k: v.copy() for k, v in arrs.items()}
                    a[kind].ravel()[i] = np.float32(x0 + sgn * step)
                    steps.append(abs(float(a[kind].ravel()[i]) - x0))
                    m = model_of(a["frame"], a["decoder"], a["pyramid"])
                    kink |= not np.array_equal(oracle.relu_pattern(m, q), pattern0)
                    vals.append(float(np.sum(dl * oracle.eval(m, q))))
                fds.append((vals[0] - vals[1]) / (steps[0] + steps[1]))
            if kink:
                continue
            fd = (4.0 * fds[1] - fds[0]) / 3.0
            an = g[kind].ravel()[i]
            assert abs(fd - an) <= 1e-6 * max(1.0, abs(an)), (kind, i, fd, an)
            done += 1
            n_out_done += kind == "decoder" and i >= dec0.size - n_out
        assert done == want[kind], (kind, done)
        if kind == "decoder":
            assert n_out_done >= 8


def test_albedo_loss_closed_form_and_differences(oracle):
    a = np.array([[1.0, 2.0, 3.0], [0.5, 0.5, 0.5]])
    t = np.array([[0.0, 0.0, 0.0], [0.5, 0.25, 1.0]], np.float32)
    L, d = oracle.albedo_loss(a, t)
    assert np.isclose(L, (1 + 4 + 9 + 0 + 0.0625 + 0.25) / 6, rtol=1e-15)
    assert np.allclose(d, 2 * (a - t) / 6, rtol=1e-15, atol=0)
    rng = np.random.default_rng(24)
    a = rng.normal(0.3, 0.5, (32, 3))
    t = rng.uniform(0, 1, (32, 3)).astype(np.float32)
    _, d = oracle.albedo_loss(a, t)
    h = 1e-6
    for i in range(0, a.size, 5):
        ap = a.copy(); ap.ravel()[i] += h
        am = a.copy(); am.ravel()[i] -= h
        fd = (oracle.albedo_loss(ap, t)[0] - oracle.albedo_loss(am, t)[0]) / (2 * h)
        assert abs(fd - d.ravel()[i]) < 1e-8


def test_albedo_targets_average_to_quadrature():
    """The training targets are unbiased: at fixed (uv, wo) their mean over
    200,000 draws matches a midpoint quadrature of Eq. 2 (integral of
    f cos(theta_i) over the hemisphere, 400 x 400 cells in (cos^2 theta, phi),
    where the cosine-weighted measure is uniform) within 4 standard errors."""
    rng = np.random.default_rng(25)
    target = W.ProceduralBRDF(np.random.default_rng(26))
    for u, v, th in ((0.3, 0.7, 0.3), (0.81, 0.12, 1.2)):
        wo = np.array([np.sin(th), 0.0, np.cos(th)])
        m = 200_000
        q = {"u": np.full(m, u, np.float32), "v": np.full(m, v, np.float32),
             "wox": np.full(m, wo[0], np.float32), "woy": np.full(m, wo[1], np.float32),
             "woz": np.full(m, wo[2], np.float32)}
        est = W.albedo_targets(rng, target, q).astype(np.float64)
        # quadrature: with s = cos^2(theta) uniform in [0,1) and phi in
        # [0, 2 pi), d(omega) cos(theta) = ds dphi / 2
        k = 400
        s = (np.arange(k) + 0.5) / k
        phi = (np.arange(k) + 0.5) / k * 2 * np.pi
        S, P = np.meshgrid(s, phi, indexing="ij")
        ct = np.sqrt(S.ravel())
        st = np.sqrt(1 - S.ravel())
        wi = np.stack([st * np.cos(P.ravel()), st * np.sin(P.ravel()), ct])
        wo_all = np.repeat(np.array([[q["wox"][0]], [q["woy"][0]], [q["woz"][0]]], np.float64), wi.shape[1], axis=1)
        f = target(np.full(wi.shape[1], float(q["u"][0])), np.full(wi.shape[1], float(q["v"][0])), wi, wo_all)
        quad = f.mean(axis=0) * np.pi       # (1/2) * (2 pi) * mean over the unit square
        se = est.std(axis=0) / np.sqrt(m)
        print(u, v, th, est.mean(axis=0), quad, se)
        assert np.all(np.abs(est.mean(axis=0) - quad) <= 4 * se + 1e-3 * quad)
