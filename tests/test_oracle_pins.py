"""Pins of the FP64 oracle against things other than itself.

Each test ties one oracle function to a closed form, an invariant, a library
routine or brute force over every texel of a tiny pyramid, chosen so that a
plausible slip (wrong texel-centre offset, swapped tap weights, wrong level
size, reversed roulette, transposed weight matrix, dropped bias, flipped
bitangent, wrong ReLU placement, wrong gradient term) fails at least one.
"""
import json
import os

import numpy as np
import pytest

import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ----------------------------------------------------------------------------
# number formats
# ----------------------------------------------------------------------------
def test_f16_decode_every_pattern(oracle):
    bits = np.arange(65536, dtype=np.uint16)
    ours = oracle.f16_bits_to_f64(bits)
    ref = bits.view(np.float16).astype(np.float64)
    nan = np.isnan(ref)
    assert np.array_equal(np.isnan(ours), nan)
    assert np.array_equal(ours[~nan], ref[~nan])


def test_f16_rounding_matches_numpy(oracle):
    rng = np.random.default_rng(1)
    x = np.concatenate([
        rng.normal(0, 1, 3000) * np.exp2(rng.uniform(-30, 17, 3000)),
        # exact ties between neighbouring binary16 values, normal and subnormal
        (np.arange(1, 400) + 0.5) * 2.0 ** -24,
        (1024 + np.arange(0, 400) + 0.5) * 2.0 ** -10,
        [65504.0, 65519.9, 65520.0, 70000.0, -65520.0, 0.0, -0.0, 2.0 ** -25, 2.0 ** -26],
    ])
    ours = oracle.f64_to_f16_bits(x)
    with np.errstate(over="ignore"):
        ref = x.astype(np.float16).view(np.uint16)
    assert np.array_equal(ours, ref)


def test_e4m3_decode_every_code(oracle):
    torch = pytest.importorskip("torch")
    codes = np.arange(256, dtype=np.uint8)
    ours = oracle.e4m3_to_f64(codes)
    ref = torch.from_numpy(codes).view(torch.float8_e4m3fn).double().numpy()
    nan = np.isnan(ref)
    assert np.array_equal(np.isnan(ours), nan)
    assert np.array_equal(ours[~nan], ref[~nan])


def test_e4m3_rounding_matches_torch_and_saturates(oracle):
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(2)
    x = np.concatenate([rng.uniform(-448, 448, 2000),
                        rng.normal(0, 1, 2000) * np.exp2(rng.uniform(-12, 8, 2000)),
                        (np.arange(8, 16) + 0.5) * 2.0 ** -3,   # ties in [1, 2)
                        (np.arange(0, 8) + 0.5) * 2.0 ** -9])   # ties among subnormals
    x = np.clip(x, -448, 448)
    ours = oracle.f64_to_e4m3(x)
    ref = torch.from_numpy(x).to(torch.float8_e4m3fn).view(torch.uint8).numpy()
    assert np.array_equal(ours, ref)
    # saturating conversion: beyond the largest finite value clamps to +-448
    assert list(oracle.e4m3_to_f64(oracle.f64_to_e4m3([500.0, 1e9, -1e9]))) == [448.0, 448.0, -448.0]


# ----------------------------------------------------------------------------
# latent filtering (Sec. 4.1)
# ----------------------------------------------------------------------------
def _tiny_model(oracle, W0, H0, L, pyr, **kw):
    dec = [(np.zeros((3, 14), np.float32), np.zeros(3, np.float32))]
    return oracle.Model(W0, H0, L, pyr, None, dec, **kw)


def _queries(u, v, lod, xi=None):
    n = len(u)
    z = np.zeros(n, np.float32)
    q = {"u": np.asarray(u, np.float32), "v": np.asarray(v, np.float32),
         "lod": np.asarray(lod, np.float32), "wix": z, "wiy": z, "wiz": z + 1,
         "wox": z, "woy": z, "woz": z + 1}
    q["xi"] = np.asarray(xi if xi is not None else np.zeros(n), np.float32)
    return q


@pytest.mark.parametrize("filt", [0, 1])
@pytest.mark.parametrize("addr", [0, 1])
def test_constant_pyramid_filters_to_constant(oracle, filt, addr):
    W0, H0, L = 16, 8, 5
    n = W.pyramid_texel_count(W0, H0, L)
    const = np.linspace(-1.5, 2.0, 8)
    pyr = np.tile(const, (n, 1)).astype(np.float32)
    m = _tiny_model(oracle, W0, H0, L, pyr, filter=filt, address=addr)
    rng = np.random.default_rng(3)
    k = 500
    q = _queries(rng.uniform(-3, 4, k), rng.uniform(-3, 4, k), rng.uniform(-2, L + 2, k), rng.random(k))
    z = oracle.latent(m, q)
    assert np.allclose(z, const[None, :], rtol=0, atol=1e-14)


def test_linear_ramp_is_reproduced_exactly(oracle):
    """Bilinear interpolation reproduces an affine function of the texel
    coordinate; texel centres at (i + 1/2)/W_l put the sample at
    x = u W_l - 1/2."""
    W0, H0, L = 32, 16, 4
    sizes = [(max(1, W0 >> l), max(1, H0 >> l)) for l in range(L)]
    pyr = []
    # dyadic slopes keep every texel exactly representable in float32
    a = np.arange(1, 9) / 8.0
    b = -np.arange(1, 9) / 16.0
    c = np.arange(-4, 4) / 4.0
    for (w, h) in sizes:
        jj, ii = np.meshgrid(np.arange(h), np.arange(w), indexing="ij")
        pyr.append(ii.reshape(-1, 1) * a + jj.reshape(-1, 1) * b + c)
    pyr = np.concatenate(pyr).astype(np.float32)
    rng = np.random.default_rng(4)
    for level, (w, h) in enumerate(sizes):
        for filt in (0, 1):
            m = _tiny_model(oracle, W0, H0, L, pyr, filter=filt)
            k = 200
            # keep x in [0, w-1] so neither wrap nor clamp takes part
            u = (rng.uniform(0, w - 1, k) + 0.5) / w
            v = (rng.uniform(0, h - 1, k) + 0.5) / h
            q = _queries(u, v, np.full(k, level), rng.random(k))
            z = oracle.latent(m, q)
            x = q["u"].astype(np.float64) * w - 0.5
            y = q["v"].astype(np.float64) * h - 0.5
            expect = x[:, None] * a + y[:, None] * b + c
            assert np.allclose(z, expect, rtol=0, atol=1e-12), (level, filt)


def _tent_periodic(d, period):
    k = np.arange(-3, 4)
    return np.maximum(0.0, 1.0 - np.abs(d[..., None] - k * period)).sum(-1)


def _brute_force_latent(pyr, W0, H0, L, u, v, lod, address):
    """Every texel of every level weighted by a tent in level space times
    a tent in each texel axis (periodic for wrap; edge-replicated for clamp)."""
    l = float(np.clip(lod, 0.0, L - 1))
    out = np.zeros(8)
    off = 0
    for lev in range(L):
        w, h = max(1, W0 >> lev), max(1, H0 >> lev)
        lam = max(0.0, 1.0 - abs(l - lev))
        tex = pyr[off:off + w * h].astype(np.float64).reshape(h, w, 8)
        off += w * h
        if lam == 0.0:
            continue
        x = float(np.float32(u)) * w - 0.5
        y = float(np.float32(v)) * h - 0.5
        if address == 0:
            wx = _tent_periodic(x - np.arange(w), w)
            wy = _tent_periodic(y - np.arange(h), h)
            out += lam * np.einsum("j,i,jic->c", wy, wx, tex)
        else:
            # the edge-replicated plane, over every lattice point near the sample
            ii = np.arange(min(-1, int(np.floor(x)) - 2), max(w + 1, int(np.floor(x)) + 3))
            jj = np.arange(min(-1, int(np.floor(y)) - 2), max(h + 1, int(np.floor(y)) + 3))
            wx = np.maximum(0.0, 1.0 - np.abs(x - ii))
            wy = np.maximum(0.0, 1.0 - np.abs(y - jj))
            sub = tex[np.clip(jj, 0, h - 1)][:, np.clip(ii, 0, w - 1)]
            out += lam * np.einsum("j,i,jic->c", wy, wx, sub)
    return out


@pytest.mark.parametrize("shape", [(4, 4, 3), (8, 8, 4), (8, 4, 4), (5, 3, 3)])
@pytest.mark.parametrize("addr", [0, 1])
def test_trilinear_equals_brute_force_over_all_texels(oracle, shape, addr):
    W0, H0, L = shape
    rng = np.random.default_rng(5)
    pyr = rng.normal(0, 0.5, (W.pyramid_texel_count(W0, H0, L), 8)).astype(np.float32)
    m = _tiny_model(oracle, W0, H0, L, pyr, filter=0, address=addr)
    k = 300
    q = _queries(rng.uniform(-2, 3, k), rng.uniform(-2, 3, k), rng.uniform(-1.5, L + 0.5, k))
    z = oracle.latent(m, q)
    for i in range(k):
        bf = _brute_force_latent(pyr, W0, H0, L, q["u"][i], q["v"][i], float(q["lod"][i]), addr)
        assert np.allclose(z[i], bf, rtol=0, atol=1e-12), i


def test_stochastic_expectation_is_trilinear(oracle):
    """Russian roulette between the two levels (Sec. 4.1): averaging over a
    midpoint grid of xi gives exactly the trilinear latent when frac(lod) is a
    multiple of the grid step."""
    W0, H0, L = 16, 16, 5
    rng = np.random.default_rng(6)
    pyr = rng.normal(0, 0.5, (W.pyramid_texel_count(W0, H0, L), 8)).astype(np.float32)
    K = 256
    mt = _tiny_model(oracle, W0, H0, L, pyr, filter=0)
    ms = _tiny_model(oracle, W0, H0, L, pyr, filter=1)
    for trial in range(20):
        lod = rng.integers(0, L - 1) + rng.integers(0, K) / K
        u, v = rng.random(2)
        zt = oracle.latent(mt, _queries([u], [v], [lod]))[0]
        xi = (np.arange(K) + 0.5) / K
        zs = oracle.latent(ms, _queries(np.full(K, u), np.full(K, v), np.full(K, lod), xi))
        assert np.allclose(zs.mean(0), zt, rtol=0, atol=1e-13)


def test_stochastic_picks_coarser_level_when_xi_below_fraction(oracle):
    W0, H0, L = 8, 8, 4
    rng = np.random.default_rng(7)
    pyr = rng.normal(0, 0.5, (W.pyramid_texel_count(W0, H0, L), 8)).astype(np.float32)
    ms = _tiny_model(oracle, W0, H0, L, pyr, filter=1)
    u, v = 0.3, 0.7
    z = oracle.latent(ms, _queries([u, u], [v, v], [1.25, 1.25], [0.1, 0.9]))
    coarse = _brute_force_latent(pyr, W0, H0, L, u, v, 2.0, 0)
    fine = _brute_force_latent(pyr, W0, H0, L, u, v, 1.0, 0)
    assert np.allclose(z[0], coarse, atol=1e-13) and np.allclose(z[1], fine, atol=1e-13)


def test_f16_pyramid_is_read_exactly(oracle):
    W0, H0, L = 8, 8, 2
    rng = np.random.default_rng(8)
    pyr = rng.normal(0, 0.5, (W.pyramid_texel_count(W0, H0, L), 8)).astype(np.float16)
    m = _tiny_model(oracle, W0, H0, L, pyr)
    # sample exactly at texel centres of level 0: the texel itself
    i, j = 3, 5
    z = oracle.latent(m, _queries([(i + 0.5) / 8], [(j + 0.5) / 8], [0.0]))[0]
    assert np.array_equal(z, pyr[j * 8 + i].astype(np.float64))


# ----------------------------------------------------------------------------
# shading frame (Sec. 4.2, Eq. 4; b = n x t / |n x t|, Sec. 9)
# ----------------------------------------------------------------------------
def test_frames_are_orthonormal_right_handed_and_match_qr(oracle):
    rng = np.random.default_rng(9)
    r = rng.normal(0, 1, (2000, 6))
    T = oracle.frame(r)
    I = np.einsum("nij,nkj->nik", T, T)
    assert np.allclose(I, np.eye(3), atol=1e-12)
    assert np.allclose(np.linalg.det(T), 1.0, atol=1e-12)
    for k in range(len(r)):
        Q, R = np.linalg.qr(np.stack([r[k, :3], r[k, 3:]], axis=1))
        q1 = Q[:, 0] * np.sign(R[0, 0])
        q2 = Q[:, 1] * np.sign(R[1, 1])
        assert np.allclose(T[k, 2], q1, atol=1e-10)   # n = normalised n_raw
        assert np.allclose(T[k, 0], q2, atol=1e-10)   # t = Gram-Schmidt of t_raw
        assert np.allclose(T[k, 1], np.cross(q1, q2), atol=1e-10)


def test_identity_frame(oracle):
    T = oracle.frame(np.array([[0, 0, 1, 1, 0, 0.0]]))[0]
    assert np.allclose(T, np.eye(3), atol=0)
    T = oracle.frame(np.array([[0, 0, 3.5, 2, 0, 1.0]]))[0]   # scale and a normal component
    assert np.allclose(T, np.eye(3), atol=1e-15)


def test_frame_rotation_equivariance(oracle):
    rng = np.random.default_rng(10)
    for _ in range(50):
        r = rng.normal(0, 1, 6)
        R, _ = np.linalg.qr(rng.normal(0, 1, (3, 3)))
        if np.linalg.det(R) < 0:
            R[:, 0] *= -1
        T = oracle.frame(r[None])[0]
        Tr = oracle.frame(np.concatenate([R @ r[:3], R @ r[3:]])[None])[0]
        w = rng.normal(0, 1, 3)
        assert np.allclose(Tr @ (R @ w), T @ w, atol=1e-12)


def test_degenerate_frames(oracle):
    T = oracle.frame(np.array([[0, 0, 0, 1, 0, 0.0]]))[0]
    assert np.allclose(T, np.eye(3))
    # tangent parallel to the normal: tangent from the normal alone
    T = oracle.frame(np.array([[0, 0, 1, 0, 0, 2.0]]))[0]
    assert np.allclose(T, np.eye(3))
    T = oracle.frame(np.array([[0, 0, -1, 0, 0, 1.0]]))[0]
    assert np.allclose(T, [[1, 0, 0], [0, -1, 0], [0, 0, -1]])
    rng = np.random.default_rng(11)
    n = rng.normal(0, 1, (200, 3))
    T = oracle.frame(np.concatenate([n, 3 * n], axis=1))
    assert np.allclose(np.einsum("nij,nkj->nik", T, T), np.eye(3), atol=1e-12)
    assert np.allclose(np.linalg.det(T), 1.0, atol=1e-12)


# ----------------------------------------------------------------------------
# MLP
# ----------------------------------------------------------------------------
@pytest.mark.parametrize("widths", [(14, 32, 32, 3), (14, 64, 64, 3), (14, 16, 16, 16, 3)])
def test_decoder_matches_numpy_matmul(oracle, widths):
    rng = np.random.default_rng(12)
    dec = W.make_mlp(rng, widths)
    m = oracle.Model(4, 4, 1, np.zeros((16, 8), np.float32), None, dec)
    x = rng.normal(0, 1, (300, widths[0]))
    a = x
    for i, (Wt, b) in enumerate(dec):
        a = a @ Wt.astype(np.float64).T + b
        if i < len(dec) - 1:
            a = np.maximum(a, 0)
    assert np.allclose(oracle.mlp(m, x), a, rtol=1e-13, atol=1e-13)


def test_identity_like_decoder_reproduces_inputs(oracle):
    I = np.eye(14, dtype=np.float32)
    dec = [(np.concatenate([I, -I]), np.zeros(28, np.float32)),
           (np.concatenate([I, -I], axis=1), np.zeros(14, np.float32))]
    m = oracle.Model(4, 4, 1, np.zeros((16, 8), np.float32), None, dec)
    x = np.random.default_rng(13).normal(0, 1, (100, 14))
    assert np.allclose(oracle.mlp(m, x), x, atol=1e-15)


@pytest.mark.parametrize("filt", [0, 1])
def test_bias_only_decoder_is_lambertian(oracle, filt):
    w = W.workload(1, scale=1 / 64)
    dec = [(np.zeros_like(Wt), np.zeros_like(b)) for Wt, b in w["model"]["decoder"]]
    rho = np.array([0.8, 0.5, 0.2], np.float32)
    dec[-1] = (dec[-1][0], rho)
    m = oracle.Model(w["W0"], w["H0"], w["L"], w["pyramid"], None, dec, filter=filt, out_cosine=True)
    q = w["queries"]
    y = oracle.eval(m, q)
    expect = rho[None, :].astype(np.float64) * np.maximum(q["wiz"].astype(np.float64), 0)[:, None]
    assert np.allclose(y, expect, rtol=0, atol=1e-15)
    m2 = oracle.Model(w["W0"], w["H0"], w["L"], w["pyramid"], None, dec, filter=filt)
    assert np.allclose(oracle.eval(m2, q), np.broadcast_to(rho.astype(np.float64), y.shape), atol=0)


def test_constant_frame_transforms_directions_by_hand(oracle):
    """Frame MLP with zero weights and bias (n_raw, t_raw) = (e_y, e_z):
    t = e_z, b = e_y x e_z = e_x, n = e_y, so T w = (w_z, w_x, w_y).  A decoder
    that copies wi' (through ReLU pairs) must return exactly that."""
    H = 16
    frame = [(np.zeros((H, 8), np.float32), np.zeros(H, np.float32)),
             (np.zeros((6, H), np.float32), np.array([0, 1, 0, 0, 0, 1], np.float32))]
    for base in (8, 11):   # wi' at inputs 8..10, wo' at 11..13
        W1 = np.zeros((6, 14), np.float32)
        for k in range(3):
            W1[2 * k, base + k] = 1
            W1[2 * k + 1, base + k] = -1
        W2 = np.zeros((3, 6), np.float32)
        for k in range(3):
            W2[k, 2 * k], W2[k, 2 * k + 1] = 1, -1
        dec = [(W1, np.zeros(6, np.float32)), (W2, np.zeros(3, np.float32))]
        w = W.workload(1, scale=1 / 64)
        m = oracle.Model(w["W0"], w["H0"], w["L"], w["pyramid"], frame, dec)
        q = w["queries"]
        y = oracle.eval(m, q)
        pre = "wi" if base == 8 else "wo"
        d = np.stack([q[pre + "z"], q[pre + "x"], q[pre + "y"]], 1).astype(np.float64)
        assert np.allclose(y, d, atol=1e-15)


def test_decoder_sees_latent_first(oracle):
    """Inputs 0..7 of the decoder are the filtered latent (input order z, wi', wo')."""
    W1 = np.zeros((16, 14), np.float32)
    for k in range(8):
        W1[2 * k, k], W1[2 * k + 1, k] = 1, -1
    W2 = np.zeros((8, 16), np.float32)
    for k in range(8):
        W2[k, 2 * k], W2[k, 2 * k + 1] = 1, -1
    w = W.workload(1, scale=1 / 64)
    m = oracle.Model(w["W0"], w["H0"], w["L"], w["pyramid"], None,
                     [(W1, np.zeros(16, np.float32)), (W2, np.zeros(8, np.float32))])
    q = w["queries"]
    x = oracle.mlp(m, np.concatenate([oracle.latent(m, q), np.zeros((len(q["u"]), 6))], 1))
    assert np.allclose(x, oracle.latent(m, q), atol=1e-15)


# ----------------------------------------------------------------------------
# gradient (reverse mode) against central finite differences
# ----------------------------------------------------------------------------
def _small_train_workload():
    rng = np.random.default_rng(14)
    W0 = H0 = 16
    L = 5
    pyr = rng.normal(0, 0.5, (W.pyramid_texel_count(W0, H0, L), 8)).astype(np.float32)
    model = W.make_model(rng, (14, 32, 32, 3), (8, 16, 6))
    q = W.uniform_queries(rng, 256, 4.0)
    return W0, H0, L, pyr, model, q, rng


def _flat_frame(fr):
    return np.concatenate([fr[0][0].ravel(), fr[0][1], fr[1][0].ravel(), fr[1][1]])


def _unflat_frame(flat, H):
    o = 0
    Wf1 = flat[o:o + H * 8].reshape(H, 8); o += H * 8
    bf1 = flat[o:o + H]; o += H
    Wf2 = flat[o:o + 6 * H].reshape(6, H); o += 6 * H
    return [(Wf1, bf1), (Wf2, flat[o:o + 6])]


def _unflat_dec(flat, widths):
    out, o = [], 0
    for a, b in zip(widths[:-1], widths[1:]):
        out.append((flat[o:o + a * b].reshape(b, a), flat[o + a * b:o + a * b + b]))
        o += a * b + b
    return out


@pytest.mark.parametrize("filt", [0, 1])
def test_gradient_matches_central_differences(oracle, filt):
    """64 random parameters (frame MLP, decoder, pyramid texels), central
    differences with h = 1e-3.  Parameters are float32, so each step is the
    realised float32 step, and the quotient divides by it exactly."""
    W0, H0, L, pyr, model, q, rng = _small_train_workload()
    dl = rng.normal(0, 1, (256, 3))
    widths = (14, 32, 32, 3)
    fr0 = _flat_frame(model["frame"]).astype(np.float32)
    dec0 = np.concatenate([np.concatenate([Wt.ravel(), b]) for Wt, b in model["decoder"]]).astype(np.float32)

    def model_of(fr, dec, p):
        return oracle.Model(W0, H0, L, p, _unflat_frame(fr, 16), _unflat_dec(dec, widths),
                            filter=filt, out_cosine=True)

    base = oracle.Model(W0, H0, L, pyr, model["frame"], model["decoder"], filter=filt, out_cosine=True)
    g = oracle.grad(base, q, dl)
    pattern0 = oracle.relu_pattern(base, q)
    h = 1e-3
    arrs = {"frame": fr0, "decoder": dec0, "pyramid": pyr}
    pools = {"frame": fr0.size, "decoder": dec0.size, "pyramid": pyr.size}
    want = {"frame": 16, "decoder": 32, "pyramid": 16}
    redraws = 0
    for kind in ("frame", "decoder", "pyramid"):
        order = rng.permutation(pools[kind])
        done = 0
        for i in order:
            if done == want[kind]:
                break
            x0 = float(arrs[kind].ravel()[i])
            kink = False
            fds = []
            for step in (h, h / 2):
                vals, steps = [], []
                for sgn in (+1, -1):
                    a = {k: v.copy() for k, v in arrs.items()}
                    a[kind].ravel()[i] = np.float32(x0 + sgn * step)
                    steps.append(abs(float(a[kind].ravel()[i]) - x0))
                    m = model_of(a["frame"], a["decoder"], a["pyramid"])
                    kink |= not np.array_equal(oracle.relu_pattern(m, q), pattern0)
                    vals.append(float(np.sum(dl * oracle.eval(m, q))))
                fds.append((vals[0] - vals[1]) / (steps[0] + steps[1]))
            if kink:       # a ReLU changes state within +-h: re-draw the parameter
                redraws += 1
                continue
            # central differences at h and h/2, Richardson-extrapolated (error
            # O(h^4)): the frame normalisation's curvature makes the O(h^2)
            # term of plain central differences visible at h = 1e-3
            fd = (4.0 * fds[1] - fds[0]) / 3.0
            an = g[kind].ravel()[i]
            assert abs(fd - an) <= 1e-6 * max(1.0, abs(an)), (kind, i, fd, an)
            done += 1
        assert done == want[kind], (kind, done, redraws)
    print(f"re-drawn for kinks: {redraws}")


def test_loss_closed_forms(oracle):
    y = np.array([[0.5, 1.0, 2.0]], np.float32)
    L0, d0 = oracle.loss(y.astype(np.float64), y)
    assert L0 == 0.0 and np.all(d0 == 0.0)
    g = np.array([[1.0, -2.0, 0.0]])
    L, d = oracle.loss(g, y)
    expect = (abs(np.log(2) - np.log(1.5)) + abs(0 - np.log(2)) + 0.01 * 2 + abs(0 - np.log(3))) / 3
    assert np.isclose(L, expect, rtol=1e-15)
    assert np.allclose(d[0], [1 / 2 / 3, -0.01 / 3, 0.0])


def test_loss_gradient_matches_central_differences(oracle):
    rng = np.random.default_rng(15)
    g = rng.normal(0.3, 0.5, (64, 3))
    y = rng.uniform(0, 1, (64, 3)).astype(np.float32)
    _, d = oracle.loss(g, y)
    h = 1e-6
    for i in range(0, g.size, 7):
        gp = g.copy(); gp.ravel()[i] += h
        gm = g.copy(); gm.ravel()[i] -= h
        fd = (oracle.loss(gp, y)[0] - oracle.loss(gm, y)[0]) / (2 * h)
        assert abs(fd - d.ravel()[i]) < 1e-8


# ----------------------------------------------------------------------------
# numbers printed in the paper
# ----------------------------------------------------------------------------
def test_paper_memory_arithmetic():
    with open(os.path.join(GOLDEN, "paper_numbers.json")) as f:
        g = json.load(f)
    t = g["latent_bytes_per_4k_tile"]
    assert 4096 * 4096 * g["latent_channels"] * 2 == t["value_bytes"]
    assert W.pyramid_texel_count(4096, 4096, 1) * 8 * 2 == 256 * 2 ** 20
