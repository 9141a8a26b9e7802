"""Pins of the oracle's reduced-precision parameter modes and helpers, from
closed forms: binary16 rounding of the parameters (Sec. 5.2: FP16 parameters
by post-training quantisation), the FP8 mode (E4M3 weights with a
power-of-two per-layer scale on the hidden -> hidden decoder layers, binary16
elsewhere), the calibration ranges and the frame condition number.  The
oracle evaluates activations in FP64 in every mode.

The models are built so that every value is known exactly: a constant FP16
pyramid (the filter then returns the constant, pinned elsewhere), directions
(0, 0, 1), no frame MLP, zero or identity weights and chosen biases; the
expected outputs are written out from the number formats' definitions."""
import numpy as np
import pytest

H = 16


def _queries(n=4):
    z = np.zeros(n, np.float32)
    one = np.ones(n, np.float32)
    return dict(u=np.linspace(0.1, 0.9, n).astype(np.float32), v=np.full(n, 0.3, np.float32),
                lod=np.full(n, 1.5, np.float32), wix=z, wiy=z, wiz=one, wox=z, woy=z, woz=one,
                xi=np.full(n, 0.5, np.float32))


def _model(oracle, b1, b2=None, c=0.5, params="master", frame=None):
    """decoder 14 -> H -> H -> 3: W1 = 0, b1 given; W2 = identity, b2 (0);
    W3 picks hidden unit 0 into every channel, b3 = 0."""
    pyr = np.full((8 * 8 + 4 * 4 + 2 * 2 + 1, 8), c, dtype=np.float16)
    W1 = np.zeros((H, 14), np.float32)
    W2 = np.eye(H, dtype=np.float32)
    W3 = np.zeros((3, H), np.float32)
    W3[:, 0] = 1.0
    dec = [(W1, np.asarray(b1, np.float32)), (W2, np.zeros(H, np.float32) if b2 is None else np.asarray(b2, np.float32)),
           (W3, np.zeros(3, np.float32))]
    return oracle.Model(8, 8, 4, pyr, frame, dec, params=params)


def _b1(v):
    b = np.zeros(H, np.float32)
    b[0] = v
    return b


@pytest.mark.parametrize("v,expect", [
    (1.0 + 2.0 ** -11, 1.0),                      # midpoint of 1 and 1 + 2^-10: ties to even
    (1.0 + 3 * 2.0 ** -11, 1.0 + 2.0 ** -9),      # midpoint of 1 + 2^-10 and 1 + 2^-9: even is the latter
    (0.1, 1638.0 / 16384.0),                      # nearest binary16 to 0.1
    (-3.0, 0.0),                                  # a negative bias, cut by the ReLU
])
def test_fp16_parameters_closed_forms(oracle, v, expect):
    """b1 carries v into hidden unit 0, which W2 = I and W3 pass to the
    output: with params="fp16" the output is v rounded to binary16; the
    activations themselves are not rounded (master parameters pass v
    through unchanged)."""
    y = oracle.eval(_model(oracle, _b1(v), params="fp16"), _queries())
    assert np.all(y == expect), (y[0], expect)
    y0 = oracle.eval(_model(oracle, _b1(v)), _queries())
    assert np.allclose(y0, max(np.float32(v), 0.0), rtol=0, atol=0)
    # a product of two binary16 values with no rounding of the activation:
    # b1 = 1 + 2^-10 (exact), W2[0][0] = 1 + 2^-10 (exact) -> h2 = (1 + 2^-10)^2
    W2 = np.eye(H, dtype=np.float32)
    W2[0, 0] = 1.0 + 2.0 ** -10
    m = _model(oracle, _b1(1.0 + 2.0 ** -10), params="fp16")
    dec = [(np.zeros((H, 14), np.float32), _b1(1.0 + 2.0 ** -10)), (W2, np.zeros(H, np.float32)),
           (m.decoder[2][0], np.zeros(3, np.float32))]
    m2 = oracle.Model(8, 8, 4, m.pyramid, None, dec, params="fp16")
    y2 = oracle.eval(m2, _queries())
    assert np.all(y2 == (1.0 + 2.0 ** -10) ** 2)


def test_fp8_weight_quantisation_closed_forms(oracle):
    """Scale: the smallest power of two s with absmax / s <= 448; codes
    E4M3(W / s), round to nearest even, 3 fraction bits, saturating."""
    W = np.array([[2.0, 1.0, 0.01, -2.0]], np.float32)
    s, deq = oracle.quantize_e4m3_layer(W)
    assert s == 2.0 ** -7                      # 2 / 448 = 2^-7.8 -> 2^-7 (2 / 2^-7 = 256 <= 448)
    # 2 / 2^-7 = 256, 1 / 2^-7 = 128, 0.01 / 2^-7 = 1.28 -> 1.25 (spacing 0.125 in [1, 2))
    codes = np.array([256.0, 128.0, 1.25, -256.0])
    assert np.all(deq.ravel() == codes * 2.0 ** -7)
    s1, deq1 = oracle.quantize_e4m3_layer(np.array([[448.0, 449.0, 1.0 + 2.0 ** -4]], np.float32))
    assert s1 == 2.0                           # 449 / 448 > 1: next power of two
    assert np.all(deq1.ravel() == np.array([448.0, 448.0, 1.0]))  # 224.5 -> 224; 0.53125 -> 0.5 (ties to even)
    s2, deq2 = oracle.quantize_e4m3_layer(np.array([[448.0, -100.0]], np.float32))
    assert s2 == 1.0 and np.all(deq2.ravel() == np.array([448.0, -96.0]))  # spacing 8 in [64, 128): 100 -> 96 (even)
    s0, deq0 = oracle.quantize_e4m3_layer(np.zeros((2, 3), np.float32))
    assert s0 == 1.0 and np.all(deq0 == 0)


def test_fp8_mode_quantises_only_hidden_to_hidden_layers(oracle):
    """params="fp8": the hidden -> hidden weights are E4M3 with their layer
    scale, every other parameter is binary16 (a swapped or shifted layer
    fails)."""
    rng = np.random.default_rng(3)
    dec = [(rng.uniform(-1, 1, (H, 14)).astype(np.float32), rng.uniform(-1, 1, H).astype(np.float32)),
           (rng.uniform(-1, 1, (H, H)).astype(np.float32), rng.uniform(-1, 1, H).astype(np.float32)),
           (rng.uniform(-1, 1, (3, H)).astype(np.float32), rng.uniform(-1, 1, 3).astype(np.float32))]
    pyr = np.full((85, 8), 0.5, dtype=np.float16)
    m8 = oracle.Model(8, 8, 4, pyr, None, dec, params="fp8")
    got = oracle.split_decoder(m8, m8.dec_params)
    s, w2 = oracle.quantize_e4m3_layer(dec[1][0])
    assert np.array_equal(got[1][0], w2.reshape(H, H))
    assert m8.weight_scales[1] == s and m8.weight_scales[0] is None and m8.weight_scales[2] is None
    for l in (0, 2):
        assert np.array_equal(got[l][0], dec[l][0].astype(np.float16).astype(np.float64))
    for l in range(3):
        assert np.array_equal(got[l][1], dec[l][1].astype(np.float16).astype(np.float64))


def test_calibration_ranges_closed_form(oracle):
    """max |input| per decoder layer: layer 0 sees (z, wi, wo) = (0.5.., 0, 0,
    1, 0, 0, 1) -> 1; layer 1 sees ReLU(b1); layer 2 sees ReLU(b2) (W2 = I
    adds ReLU(b1) on the diagonal)."""
    b1 = np.linspace(-1.0, 3.0, H).astype(np.float32)
    b2 = np.full(H, -10.0, np.float32)
    b2[5] = 7.5
    m = _model(oracle, b1, b2=b2, c=0.75)
    amax = oracle.decoder_input_absmax(m, _queries())
    assert amax[0] == 1.0
    assert amax[1] == np.float32(3.0)
    relu_b1 = np.maximum(b1.astype(np.float64), 0)
    assert amax[2] == np.max(np.maximum(relu_b1 + b2, 0))


@pytest.mark.parametrize("n_raw,t_raw,kappa", [
    ((0.0, 0.0, 1.0), (1.0, 0.0, 1.0), np.sqrt(2.0)),   # 45 degrees: 1 / sin
    ((0.0, 0.0, 2.0), (0.0, 3.0, 0.0), 1.0),            # orthogonal
    ((0.0, 0.0, 1.0), (0.5, 0.0, 0.5 * np.sqrt(3.0)), 2.0),  # 30 degrees
])
def test_frame_condition_closed_forms(oracle, n_raw, t_raw, kappa):
    """Frame MLP with zero weights: r = (n_raw, t_raw) comes from the output
    bias alone, each component's magnitude sum is its own magnitude, so kappa
    = 1 / sin(angle(n_raw, t_raw))."""
    frame = [(np.zeros((16, 8), np.float32), np.zeros(16, np.float32)),
             (np.zeros((6, 16), np.float32), np.array(n_raw + t_raw, np.float32))]
    m = _model(oracle, _b1(1.0), frame=frame)
    k = oracle.frame_condition(m, _queries())
    assert np.allclose(k, kappa, rtol=1e-6)


@pytest.mark.parametrize("cosine", [False, True])
def test_direction_gain_matches_finite_differences(oracle, cosine):
    """direction_gain is the sum over the six direction inputs of
    |dy/dx| through the ReLU pattern: against central differences of the
    oracle's decoder alone (no frame MLP, so the inputs are (z, wi, wo)),
    with two step sizes that must agree (a pair straddling a ReLU kink is
    skipped); with the cosine factor every channel scales by max(0, wi.z)."""
    import workloads as W
    rng = W.rng_streams(4242, 3)
    pyr = W.make_pyramid(rng[0], 32, 32, 6, dtype=np.float16)
    model = W.make_model(rng[1], (14, 32, 32, 3), None)
    om = oracle.Model(32, 32, 6, pyr, model["frame"], model["decoder"], out_cosine=cosine)
    q = W.uniform_queries(rng[2], 400, 5.0)
    gain = oracle.direction_gain(om, q)
    z = oracle.latent(om, q)
    x = np.concatenate([z, np.stack([q["wix"], q["wiy"], q["wiz"], q["wox"], q["woy"], q["woz"]], 1)], 1)
    x = x.astype(np.float64)

    def fd(h):
        J = np.zeros((len(x), 3, 6))
        for k in range(6):
            xp, xm = x.copy(), x.copy()
            xp[:, 8 + k] += h
            xm[:, 8 + k] -= h
            J[:, :, k] = (oracle.mlp(om, xp)[:, :3] - oracle.mlp(om, xm)[:, :3]) / (2 * h)
        return np.abs(J).sum(axis=2)

    g1, g2 = fd(1e-6), fd(2.5e-7)
    cosf = np.maximum(q["wiz"].astype(np.float64), 0.0)[:, None] if cosine else 1.0
    g1, g2 = g1 * cosf, g2 * cosf
    scale = np.maximum(np.abs(g1), 1e-3)
    smooth = (np.abs(g1 - g2) / scale < 1e-6).all(axis=1)
    assert smooth.mean() > 0.95
    assert np.allclose(gain[smooth], g1[smooth], rtol=1e-6, atol=1e-9)
    assert (gain > 0).any()


def test_gain_bound_reduces_to_unit_gain_form(oracle):
    """parity's band bound with gain = den / 2 equals the bound without a
    gain; a larger gain loosens only the queries beyond kappa = 50."""
    rng = np.random.default_rng(5)
    o = rng.normal(size=(6, 3)) + 2.0
    kappa = np.array([1.0, 10.0, 60.0, 100.0, 1000.0, 5e4])
    tau = float(np.sqrt(np.mean(o * o)))
    den = np.maximum(np.abs(o), tau)
    eps = 2.0 ** -18
    # errors placed exactly at 0.99 of the unit-gain bound
    b = np.where(kappa[:, None] <= 50, 2e-3, 2e-3 + eps * (1 + 2 * kappa[:, None]) * 0.5)
    g = o + 0.99 * b * den
    ok0, st0 = oracle.parity(g, o, kappa, 2e-3)
    ok1, st1 = oracle.parity(g, o, kappa, 2e-3, gain=den / 2)
    assert ok0 and ok1 and abs(st0["worst_over_bound"] - st1["worst_over_bound"]) < 1e-12
    g2 = o + 1.01 * b * den
    assert not oracle.parity(g2, o, kappa, 2e-3)[0]
    ok3, _ = oracle.parity(g2, o, kappa, 2e-3, gain=np.where(kappa[:, None] > 50, den, den / 2))
    assert not ok3  # the well-conditioned rows still fail at 1.01 tol
    g4 = np.where(kappa[:, None] > 50, g2, g)
    assert oracle.parity(g4, o, kappa, 2e-3, gain=den)[0]
