"""Pins of the oracle's reduced-precision emulation and of its helpers, from
closed forms: the rounding of decoder inputs to FP16 (Sec. 5.2: FP16
parameters and, on tensor cores, FP16 operands, Sec. 7.2) and to E4M3 with a
static scale, the list of valid results at a rounding midpoint, the FP8 weight
quantisation, the calibration ranges and the frame condition number.

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


def _model(oracle, b1, b2=None, c=0.5, params="master", act_round=0, act_scale=None, frame=None):
    """decoder 14 -> H -> H -> 3: W1 = 0, b1 given; W2 = identity, b2 (0);
    W3 picks hidden unit 0 into every channel, b3 = 0."""
    pyr = np.full((8 * 8 + 4 * 4 + 2 * 2 + 1, 8), c, dtype=np.float16)
    W1 = np.zeros((H, 14), np.float32)
    W2 = np.eye(H, dtype=np.float32)
    W3 = np.zeros((3, H), np.float32)
    W3[:, 0] = 1.0
    dec = [(W1, np.asarray(b1, np.float32)), (W2, np.zeros(H, np.float32) if b2 is None else np.asarray(b2, np.float32)),
           (W3, np.zeros(3, np.float32))]
    return oracle.Model(8, 8, 4, pyr, frame, dec, params=params, act_round=act_round, act_scale=act_scale)


def _b1(v):
    b = np.zeros(H, np.float32)
    b[0] = v
    return b


@pytest.mark.parametrize("v,expect", [
    (1.0 + 2.0 ** -11, 1.0),                      # midpoint of 1 and 1 + 2^-10: ties to even
    (1.0 + 3 * 2.0 ** -11, 1.0 + 2.0 ** -9),      # midpoint of 1 + 2^-10 and 1 + 2^-9: even is the latter
    (0.1, 1638.0 / 16384.0),                      # nearest binary16 to 0.1
    (70000.0, np.inf),                            # beyond 65504 + half a step: overflow
    (-3.0, 0.0),                                  # ReLU before the rounding
])
def test_fp16_operand_rounding_closed_forms(oracle, v, expect):
    m = _model(oracle, _b1(v), act_round=oracle.ROUND_FP16)
    y = oracle.eval(m, _queries())
    assert np.all(y == expect), (y[0], expect)
    # without operand rounding the value passes through unchanged
    y0 = oracle.eval(_model(oracle, _b1(v)), _queries())
    assert np.allclose(y0, max(np.float32(v), 0.0), rtol=0, atol=0)


@pytest.mark.parametrize("v,scale,expect", [
    (1.0 + 2.0 ** -4, 1.0, 1.0),        # midpoint of 1 and 1.125 (3 fraction bits): ties to even
    (1.1875, 1.0, 1.25),                # midpoint of 1.125 and 1.25: even is 1.25
    (2.125, 2.0, 2.0),                  # the same decision after the scale (2.125 / 2 = 1.0625)
    (500.0, 1.0, 448.0),                # saturates at the largest finite E4M3
    (0.001, 1.0, 2.0 ** -9),            # nearest subnormal (spacing 2^-9)
    (0.0009, 1.0, 0.0),                 # below half the smallest subnormal
])
def test_fp8_operand_rounding_closed_forms(oracle, v, scale, expect):
    s = np.full(3, scale)
    m = _model(oracle, _b1(v), params="fp8", act_round=oracle.ROUND_FP8, act_scale=s)
    y = oracle.eval(m, _queries())
    # identity and pick weights dequantise to 1 within FP32 rounding of 1/448
    assert np.allclose(y, expect, rtol=2e-7, atol=0), (y[0], expect)


def test_fp8_layer_input_zero_is_not_rounded_away(oracle):
    """z and the directions are layer-0 inputs: with an exact constant pyramid
    (0.5) and directions (0, 0, 1) the E4M3 codes are exact."""
    W1 = np.zeros((H, 14), np.float32)
    W1[0, 0] = 1.0       # h1[0] = z0
    W1[1, 10] = 1.0      # h1[1] = wi_z
    pyr = np.full((85, 8), 0.5, dtype=np.float16)
    W3 = np.zeros((3, H), np.float32)
    W3[0, 0] = 1.0
    W3[1, 1] = 1.0
    dec = [(W1, np.zeros(H, np.float32)), (np.eye(H, dtype=np.float32), np.zeros(H, np.float32)),
           (W3, np.zeros(3, np.float32))]
    m = oracle.Model(8, 8, 4, pyr, None, dec, params="fp8", act_round=oracle.ROUND_FP8, act_scale=np.ones(3))
    y = oracle.eval(m, _queries())
    assert np.allclose(y[:, 0], 0.5, rtol=3e-7) and np.allclose(y[:, 1], 1.0, rtol=3e-7) and np.all(y[:, 2] == 0)


def test_fp8_weight_quantisation_closed_forms(oracle):
    W = np.array([[2.0, 1.0, 0.01, -2.0]], np.float32)
    s, deq = oracle.quantize_e4m3_layer(W)
    assert s == np.float32(2.0) / np.float32(448.0)
    codes = np.array([448.0, 224.0, 2.25, -448.0])   # 0.01 / s = 2.24 -> 2.25 (spacing 0.25 in [2, 4))
    assert np.allclose(deq.ravel(), codes * float(s), rtol=0, atol=0)
    s0, deq0 = oracle.quantize_e4m3_layer(np.zeros((2, 3), np.float32))
    assert s0 == 1.0 and np.all(deq0 == 0)


def test_alternatives_at_an_exact_midpoint(oracle):
    """One activation exactly at a binary16 midpoint: both neighbours are
    valid results; away from any midpoint there is a single result."""
    m = _model(oracle, _b1(1.0 + 2.0 ** -11), act_round=oracle.ROUND_FP16)
    alts, nalt, nsites = oracle.eval_alternatives(m, _queries())
    assert np.all(nsites == 1) and np.all(nalt == 2)
    got = np.sort(alts[:, :2, 0], axis=1)
    assert np.all(got == np.array([1.0, 1.0 + 2.0 ** -10]))
    assert np.all(alts[:, 0, 0] == 1.0)  # nominal first
    m2 = _model(oracle, _b1(1.0 + 2.0 ** -12), act_round=oracle.ROUND_FP16)
    alts2, nalt2, _ = oracle.eval_alternatives(m2, _queries())
    assert np.all(nalt2 == 1) and np.all(alts2[:, 0, 0] == 1.0)


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
