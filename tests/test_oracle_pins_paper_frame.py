"""Pins of the oracle's paper-form shading frames (Sec. 4.2, Eq. 4: one
linear layer gives N = 2 normals and tangents, each normalised but not
orthogonalised, b = n x t / |n x t| as Sec. 9 states) and of the 20-input
decoder that reads (z, T wi, T wo), against frames worked out by hand."""
import numpy as np
import pytest

S2 = 1.0 / np.sqrt(2.0)
N_IN = 20


def _model(oracle, r12, W1, b1=None, H=32, n_hidden=2):
    """Frame layer with zero weights and output bias r12; decoder 20 -> H ->
    ... -> 3 with first-layer weights W1 [H][20], identity hidden layers and
    an output layer that copies hidden units 0..2."""
    pyr = np.full((85, 8), 0.5, np.float16)
    frame = [(np.zeros((12, 8), np.float32), np.asarray(r12, np.float32))]
    dec = [(np.asarray(W1, np.float32), np.zeros(H, np.float32) if b1 is None else np.asarray(b1, np.float32))]
    for _ in range(n_hidden - 1):
        dec.append((np.eye(H, dtype=np.float32), np.zeros(H, np.float32)))
    W3 = np.zeros((3, H), np.float32)
    W3[0, 0] = W3[1, 1] = W3[2, 2] = 1.0
    dec.append((W3, np.zeros(3, np.float32)))
    return oracle.Model(8, 8, 4, pyr, frame, dec)


def _queries(wi, wo):
    wi = np.asarray(wi, np.float32)
    wo = np.asarray(wo, np.float32)
    n = len(wi)
    return dict(u=np.full(n, 0.2, np.float32), v=np.full(n, 0.7, np.float32), lod=np.full(n, 0.5, np.float32),
                wix=wi[:, 0].copy(), wiy=wi[:, 1].copy(), wiz=wi[:, 2].copy(), wox=wo[:, 0].copy(),
                woy=wo[:, 1].copy(), woz=wo[:, 2].copy(), xi=np.zeros(n, np.float32))


def _pick(cols, H=32):
    """First-layer weights copying decoder inputs `cols` into hidden units
    0..2 (inputs: 0..7 z, 8..13 T wi, 14..19 T wo)."""
    W = np.zeros((H, N_IN), np.float32)
    for j, c in enumerate(cols):
        W[j, c] = 1.0
    return W


# frame 1: n = (0, 0, 2), t = (3, 0, 0)  -> (t, b, n) = (x, y, z)
# frame 2: n = (0, 5, 0), t = (0, 1, 1)  -> n = y, t = (y + z)/sqrt2, b = n x t / |n x t| = x
R12 = [0, 0, 2, 3, 0, 0, 0, 5, 0, 0, 1, 1]


def _expected(w):
    """T w for the two hand-built frames: (t1, b1, n1, t2, b2, n2) . w."""
    x, y, z = w[:, 0].astype(np.float64), w[:, 1].astype(np.float64), w[:, 2].astype(np.float64)
    return np.stack([x, y, z, (y + z) * S2, x, y], axis=1)


@pytest.mark.parametrize("n_hidden", [2, 3])
def test_paper_frames_transform_directions_by_hand(oracle, n_hidden):
    rng = np.random.default_rng(4)
    wi = rng.normal(size=(6, 3))
    wi[:, 2] = np.abs(wi[:, 2])
    wi /= np.linalg.norm(wi, axis=1, keepdims=True)
    wo = rng.normal(size=(6, 3))
    wo[:, 2] = np.abs(wo[:, 2])
    wo /= np.linalg.norm(wo, axis=1, keepdims=True)
    q = _queries(wi, wo)
    ei = _expected(np.stack([q["wix"], q["wiy"], q["wiz"]], 1))
    eo = _expected(np.stack([q["wox"], q["woy"], q["woz"]], 1))
    # ReLU hidden layers: shift by +2 so that every picked value stays positive
    for cols, ref in (((8, 9, 10), ei[:, :3]), ((11, 12, 13), ei[:, 3:]), ((14, 15, 16), eo[:, :3]),
                      ((17, 18, 19), eo[:, 3:])):
        b1 = np.zeros(32, np.float32)
        b1[:3] = 2.0
        y = oracle.eval(_model(oracle, R12, _pick(cols), b1=b1, n_hidden=n_hidden), q)
        assert np.allclose(y - 2.0, ref, atol=1e-12), cols


def test_decoder_reads_latent_first(oracle):
    q = _queries([[0, 0, 1]], [[0, 0, 1]])
    b1 = np.zeros(32, np.float32)
    y = oracle.eval(_model(oracle, R12, _pick((0, 3, 7)), b1=b1), q)
    assert np.allclose(y, 0.5)  # constant pyramid 0.5 in every channel


def test_orthonormal_case_equals_gram_schmidt_form(oracle):
    """With n and t orthonormal the paper's frame equals the Gram-Schmidt
    frame of the MLP form: a decoder reading only frame 1 gives the same
    output as the 14-input decoder of the MLP form with the same frame."""
    n1 = np.array([0.0, 0.6, 0.8])
    t1 = np.array([1.0, 0.0, 0.0])
    r12 = np.concatenate([n1, t1, [0, 0, 1], [1, 0, 0]])
    rng = np.random.default_rng(5)
    H = 32
    Wd = rng.normal(size=(H, 14)).astype(np.float32)
    W20 = np.zeros((H, 20), np.float32)
    W20[:, :8] = Wd[:, :8]
    W20[:, 8:11] = Wd[:, 8:11]     # T1 wi
    W20[:, 14:17] = Wd[:, 11:14]   # T1 wo
    b1 = rng.normal(size=H).astype(np.float32)
    W2 = rng.normal(size=(H, H)).astype(np.float32) * 0.2
    W3 = rng.normal(size=(3, H)).astype(np.float32)
    pyr = np.random.default_rng(6).normal(size=(85, 8)).astype(np.float16)
    paper = oracle.Model(8, 8, 4, pyr, [(np.zeros((12, 8), np.float32), r12.astype(np.float32))],
                         [(W20, b1), (W2, np.zeros(H, np.float32)), (W3, np.zeros(3, np.float32))])
    mlp = oracle.Model(8, 8, 4, pyr, [(np.zeros((16, 8), np.float32), np.zeros(16, np.float32)),
                                      (np.zeros((6, 16), np.float32), np.concatenate([n1, t1]).astype(np.float32))],
                       [(Wd, b1), (W2, np.zeros(H, np.float32)), (W3, np.zeros(3, np.float32))])
    wi = rng.normal(size=(50, 3))
    wi /= np.linalg.norm(wi, axis=1, keepdims=True)
    wo = rng.normal(size=(50, 3))
    wo /= np.linalg.norm(wo, axis=1, keepdims=True)
    q = _queries(wi, wo)
    q["u"] = rng.random(50).astype(np.float32)
    q["v"] = rng.random(50).astype(np.float32)
    assert np.allclose(oracle.eval(paper, q), oracle.eval(mlp, q), rtol=1e-12, atol=1e-12)


def test_degenerate_paper_frames(oracle):
    """n_raw = 0 -> n = (0,0,1); n parallel to t -> t from n (Duff et al.),
    an orthonormal right-handed frame either way."""
    q = _queries([[0.3, -0.4, np.sqrt(0.75)]], [[0, 0, 1]])
    for r12 in ([0, 0, 0, 1, 0, 0, 0, 0, 1, 0, 0, 3], [0, 2, 0, 0, -1, 0, 0, 0, 1, 1, 0, 0]):
        cols = (8, 9, 10)
        b1 = np.zeros(32, np.float32)
        b1[:3] = 2.0
        y = oracle.eval(_model(oracle, r12, _pick(cols), b1=b1), q) - 2.0
        # the transformed wi has the norm of wi
        assert np.isclose(np.linalg.norm(y[0]), 1.0, atol=1e-12)
    k = oracle.frame_condition(_model(oracle, R12, _pick((8, 9, 10))), q)
    # frame 2 has sin(n, t) = 1/sqrt(2): kappa = sqrt(2) (zero weights, so each
    # raw vector's magnitude sum is its norm)
    assert np.isclose(k[0], np.sqrt(2.0), rtol=1e-12)


def test_reverse_mode_of_paper_form_is_refused(oracle):
    q = _queries([[0, 0, 1]], [[0, 0, 1]])
    with pytest.raises(NotImplementedError):
        oracle.grad(_model(oracle, R12, _pick((8, 9, 10))), q, np.ones((1, 3)))
