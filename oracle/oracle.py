"""Python front end of the FP64 CPU oracle (oracle/nam_oracle.c).

TEST INFRASTRUCTURE: only the tests, the smoke check and the benchmark's
CPU-baseline leg import this module.  It builds the C library with gcc on
first use (or from `build()`), and marshals numpy arrays into it.  It never
imports the CUDA package, and the CUDA package never imports it.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "nam_oracle.c")
_LIB = os.path.join(_HERE, "_build", "liboracle.so")
_lib = None

FILTER_TRILINEAR, FILTER_STOCHASTIC = 0, 1
ADDRESS_WRAP, ADDRESS_CLAMP = 0, 1
MAXL = 8


def build(force: bool = False) -> str:
    """Compile liboracle.so with gcc (plain C, -O2, no fast-math)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        os.makedirs(os.path.dirname(_LIB), exist_ok=True)
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fno-fast-math",
                               "-ffp-contract=off", "-o", tmp, _SRC, "-lm", "-lpthread"])
        os.replace(tmp, _LIB)
    return _LIB


class _Model(C.Structure):
    _fields_ = [("W0", C.c_int32), ("H0", C.c_int32), ("L", C.c_int32), ("C", C.c_int32),
                ("latent_f16", C.c_int32), ("address", C.c_int32), ("filter", C.c_int32),
                ("out_cosine", C.c_int32), ("frame_hidden", C.c_int32), ("n_layers", C.c_int32),
                ("widths", C.c_int32 * (MAXL + 1)),
                ("pyramid", C.c_void_p), ("frame_params", C.c_void_p),
                ("dec_params", C.c_void_p), ("frame_form", C.c_int32)]


class _Queries(C.Structure):
    # "z" (float64 [n][8], optional): latents given directly (encoder phase,
    # Sec. 5.1); the other fields are float32 arrays
    _fields_ = [(k, C.c_void_p) for k in ("u", "v", "lod", "wix", "wiy", "wiz", "wox", "woy", "woz", "xi", "z")]


def lib():
    global _lib
    if _lib is None:
        _lib = C.CDLL(build())
        d, p, i64, u16, u8 = C.c_double, C.c_void_p, C.c_int64, C.c_uint16, C.c_uint8
        _lib.orc_f16_to_f64.restype = d; _lib.orc_f16_to_f64.argtypes = [u16]
        _lib.orc_f64_to_f16.restype = u16; _lib.orc_f64_to_f16.argtypes = [d]
        _lib.orc_round_f16.restype = d; _lib.orc_round_f16.argtypes = [d]
        _lib.orc_e4m3_to_f64.restype = d; _lib.orc_e4m3_to_f64.argtypes = [u8]
        _lib.orc_qtanh.restype = d; _lib.orc_qtanh.argtypes = [d]
        _lib.orc_qsinh.restype = d; _lib.orc_qsinh.argtypes = [d]
        _lib.orc_proxy_activate.argtypes = [p, p]
        _lib.orc_proxy_pdf_h.restype = d; _lib.orc_proxy_pdf_h.argtypes = [p, p]
        _lib.orc_proxy_pdf.restype = d; _lib.orc_proxy_pdf.argtypes = [p, p, p]
        _lib.orc_proxy_sample.argtypes = [p, p, p, p, p]
        _lib.orc_sampler_params.argtypes = [p, p, p, i64, p]
        _lib.orc_sampler_pdf.argtypes = [p, p, p, i64, p]
        _lib.orc_sampler_sample.argtypes = [p, p, p, i64, p, p, p]
        _lib.orc_proxy_pdf_batch.argtypes = [p, p, p, i64, p]
        _lib.orc_proxy_pdf_h_batch.argtypes = [p, p, i64, p]
        _lib.orc_f64_to_e4m3.restype = u8; _lib.orc_f64_to_e4m3.argtypes = [d]
        _lib.orc_round_e4m3.restype = d; _lib.orc_round_e4m3.argtypes = [d]
        _lib.orc_quantize_e4m3_layer.argtypes = [p, i64, p, p]
        _lib.orc_latent_batch.argtypes = [p, p, i64, p]
        _lib.orc_frame_batch.argtypes = [p, i64, p]
        _lib.orc_mlp_batch.argtypes = [p, p, i64, p]
        _lib.orc_eval.argtypes = [p, p, i64, p, C.c_int]
        _lib.orc_decoder_input_absmax.argtypes = [p, p, i64, p]
        _lib.orc_loss.restype = d; _lib.orc_loss.argtypes = [p, p, i64, p]
        _lib.orc_albedo_loss.restype = d; _lib.orc_albedo_loss.argtypes = [p, p, i64, p]
        _lib.orc_grad.argtypes = [p, p, i64, p, p, p, p, p]
        _lib.orc_relu_pattern.argtypes = [p, p, i64, p]
        _lib.orc_frame_condition.argtypes = [p, p, i64, p]
        _lib.orc_direction_gain.argtypes = [p, p, i64, p]
    return _lib


def _ptr(a):
    return a.ctypes.data_as(C.c_void_p) if a is not None else None


# ----------------------------------------------------------------------------
# number formats
# ----------------------------------------------------------------------------
def f16_bits_to_f64(bits):
    L = lib()
    return np.array([L.orc_f16_to_f64(int(b)) for b in np.asarray(bits).ravel()])


def round_f16(x):
    L = lib()
    x = np.asarray(x, dtype=np.float64)
    return np.array([L.orc_round_f16(float(v)) for v in x.ravel()]).reshape(x.shape)


def f64_to_f16_bits(x):
    L = lib()
    x = np.asarray(x, dtype=np.float64)
    return np.array([L.orc_f64_to_f16(float(v)) for v in x.ravel()], dtype=np.uint16).reshape(x.shape)


def e4m3_to_f64(codes):
    L = lib()
    return np.array([L.orc_e4m3_to_f64(int(b)) for b in np.asarray(codes).ravel()])


def f64_to_e4m3(x):
    L = lib()
    x = np.asarray(x, dtype=np.float64)
    return np.array([L.orc_f64_to_e4m3(float(v)) for v in x.ravel()], dtype=np.uint8).reshape(x.shape)


def quantize_e4m3_layer(W):
    """(scale, dequantised weights) of one layer: power-of-two scale, codes
    E4M3(W / scale)."""
    W = np.ascontiguousarray(W, dtype=np.float32)
    s = np.zeros(1, dtype=np.float32)
    out = np.zeros(W.shape, dtype=np.float64)
    lib().orc_quantize_e4m3_layer(_ptr(W), W.size, _ptr(s), _ptr(out))
    return float(s[0]), out


# ----------------------------------------------------------------------------
# model
# ----------------------------------------------------------------------------
class Model:
    """A neural material as the oracle sees it.

    pyramid: [texels, 8] float16 or float32; frame: None or [(Wf1,bf1),(Wf2,bf2)];
    decoder: [(W,b), ...] with W [out][in].  `params` selects the parameter
    values: "master" (as given), "fp16" (each rounded to binary16 by the
    oracle's own rounding), "fp8" (as "fp16", except the weights of the
    hidden -> hidden decoder layers: E4M3 with a power-of-two per-layer scale).
    Activations are always evaluated in FP64.
    """

    def __init__(self, W0, H0, L, pyramid, frame, decoder, *, filter=FILTER_TRILINEAR,
                 address=ADDRESS_WRAP, out_cosine=False, params="master"):
        self.W0, self.H0, self.L = W0, H0, L
        self.pyramid = np.ascontiguousarray(pyramid)
        assert self.pyramid.shape[1] == 8
        f16 = self.pyramid.dtype == np.float16
        if f16:
            self._pyr = self.pyramid.view(np.uint16)
        else:
            self._pyr = np.ascontiguousarray(self.pyramid, dtype=np.float32)
        self.frame = frame
        self.decoder = decoder
        self.widths = [decoder[0][0].shape[1]] + [W.shape[0] for W, _ in decoder]
        self.weight_scales = None
        # frame: [(Wf1, bf1), (Wf2, bf2)] = the MLP form 8 -> h -> 6 with
        # Gram-Schmidt; [(Wf, bf)] with Wf [12][8] = the paper's form (one
        # linear layer, two frames, decoder input width 20)
        self.frame_form = 1 if (frame is not None and len(frame) == 1) else 0
        if frame is not None:
            fp = np.concatenate([np.concatenate([W.ravel(), b]) for W, b in frame])
            fp = fp.astype(np.float64)
            if params in ("fp16", "fp8"):
                fp = round_f16(fp)
        else:
            fp = None
        chunks = []
        scales = []
        for l, (W, b) in enumerate(decoder):
            hidden_to_hidden = 0 < l < len(decoder) - 1
            if params == "fp8" and hidden_to_hidden:
                s, Wd = quantize_e4m3_layer(W)
                scales.append(s)
                chunks += [Wd.ravel(), round_f16(b.astype(np.float64))]
            elif params in ("fp16", "fp8"):
                scales.append(None)
                chunks += [round_f16(W.astype(np.float64)).ravel(), round_f16(b.astype(np.float64))]
            else:
                chunks += [W.astype(np.float64).ravel(), b.astype(np.float64)]
        if params == "fp8":
            self.weight_scales = scales
        self.frame_params = fp
        self.dec_params = np.ascontiguousarray(np.concatenate(chunks))
        s = _Model()
        s.W0, s.H0, s.L, s.C = W0, H0, L, 8
        s.latent_f16 = int(f16)
        s.address = address
        s.filter = filter
        s.out_cosine = int(bool(out_cosine))
        s.frame_hidden = 0 if (frame is None or self.frame_form == 1) else frame[0][0].shape[0]
        s.frame_form = self.frame_form
        s.n_layers = len(decoder)
        for i, w in enumerate(self.widths):
            s.widths[i] = w
        s.pyramid = self._pyr.ctypes.data
        s.frame_params = None if fp is None else fp.ctypes.data
        s.dec_params = self.dec_params.ctypes.data
        self._s = s

    @classmethod
    def from_workload(cls, w, **kw):
        m = w["model"]
        return cls(w["W0"], w["H0"], w["L"], w["pyramid"], m["frame"], m["decoder"], **kw)

    def texel_count(self):
        return self.pyramid.shape[0]

    def n_frame_params(self):
        return 0 if self.frame_params is None else self.frame_params.size

    def n_dec_params(self):
        return self.dec_params.size


class _QueryView:
    def __init__(self, q, n):
        self.arrays = {}
        for k in _Queries._fields_:
            name = k[0]
            a = q.get(name)
            if a is None:
                self.arrays[name] = None
                continue
            a = np.ascontiguousarray(a, dtype=np.float64 if name == "z" else np.float32)
            assert a.shape[0] >= n
            self.arrays[name] = a
        s = _Queries()
        for name, a in self.arrays.items():
            setattr(s, name, None if a is None else a.ctypes.data)
        self.s = s


def _nq(q):
    return int(q["u"].shape[0])


def eval(model: Model, q, nthreads: int | None = None) -> np.ndarray:
    """[n, 3] RGB, or [n, 6] (RGB, albedo RGB) for a decoder with the albedo
    head (6 outputs; the cosine factor applies to the RGB only)."""
    n = _nq(q)
    out = np.zeros((n, model.widths[-1]), dtype=np.float64)
    if n == 0:
        return out
    qv = _QueryView(q, n)
    if nthreads is None:
        nthreads = os.cpu_count() or 1
    lib().orc_eval(C.byref(model._s), C.byref(qv.s), n, _ptr(out), nthreads)
    return out


def latent(model: Model, q) -> np.ndarray:
    n = _nq(q)
    out = np.zeros((n, 8), dtype=np.float64)
    qv = _QueryView(q, n)
    lib().orc_latent_batch(C.byref(model._s), C.byref(qv.s), n, _ptr(out))
    return out


def frame(r) -> np.ndarray:
    """[n,6] raw (n_raw, t_raw) -> [n,3,3] T with rows t, b, n."""
    r = np.ascontiguousarray(r, dtype=np.float64).reshape(-1, 6)
    out = np.zeros((r.shape[0], 9), dtype=np.float64)
    lib().orc_frame_batch(_ptr(r), r.shape[0], _ptr(out))
    return out.reshape(-1, 3, 3)


def mlp(model: Model, x) -> np.ndarray:
    x = np.ascontiguousarray(x, dtype=np.float64)
    n = x.shape[0]
    out = np.zeros((n, model.widths[-1]), dtype=np.float64)
    lib().orc_mlp_batch(C.byref(model._s), _ptr(x), n, _ptr(out))
    return out


def decoder_input_absmax(model: Model, q) -> np.ndarray:
    n = _nq(q)
    out = np.zeros(len(model.decoder), dtype=np.float64)
    qv = _QueryView(q, n)
    lib().orc_decoder_input_absmax(C.byref(model._s), C.byref(qv.s), n, _ptr(out))
    return out


def relu_pattern(model: Model, q) -> np.ndarray:
    """Per-query hash of the on/off state of every ReLU the query passes."""
    n = _nq(q)
    out = np.zeros(n, dtype=np.uint64)
    qv = _QueryView(q, n)
    lib().orc_relu_pattern(C.byref(model._s), C.byref(qv.s), n, _ptr(out))
    return out


def frame_condition(model: Model, q) -> np.ndarray:
    """Per-query condition number of the frame step (1 without a frame MLP)."""
    n = _nq(q)
    out = np.ones(n, dtype=np.float64)
    if n:
        qv = _QueryView(q, n)
        lib().orc_frame_condition(C.byref(model._s), C.byref(qv.s), n, _ptr(out))
    return out


def direction_gain(model: Model, q) -> np.ndarray:
    """Per query and RGB channel: sum over the decoder's direction inputs of
    |d y / d x| through the query's ReLU pattern (with the cosine factor):
    a first-order bound on how far y moves per unit of direction error."""
    n = _nq(q)
    out = np.zeros((n, 3), dtype=np.float64)
    if n:
        qv = _QueryView(q, n)
        lib().orc_direction_gain(C.byref(model._s), C.byref(qv.s), n, _ptr(out))
    return out


def band_gain(model: Model, q, kappa, kappa_well=50.0) -> np.ndarray:
    """direction_gain for the queries beyond kappa_well (zeros elsewhere,
    where parity does not read it)."""
    kappa = np.asarray(kappa)
    out = np.zeros((len(kappa), 3), dtype=np.float64)
    idx = np.nonzero(kappa > kappa_well)[0]
    if len(idx):
        out[idx] = direction_gain(model, {k: np.asarray(v)[idx] for k, v in q.items() if v is not None})
    return out


def parity(g, o, kappa, tol, gain=None, kappa_well=50.0, eps=2.0 ** -18, tau=None):
    """Element-wise parity with a conditioning-aware bound.

    rel = |g - o| / max(|o|, tau) per channel, tau = RMS of o.  Queries whose
    frame condition number kappa is at most kappa_well must meet `tol`.
    Beyond it the bound adds the frame arithmetic's error as the decoder
    sees it: the raw frame outputs carry a relative error of at most eps
    (measured against the sum of their terms' magnitudes, which kappa
    includes), which moves the frame, and so every transformed direction, by
    at most (1 + 2 kappa) eps; the decoder turns that into at most
    gain * (1 + 2 kappa) eps on the output (`gain` from direction_gain).
    Without `gain` the decoder's gain relative to max(|o|, tau) is taken as
    1/2.  `tau` overrides the RMS floor (a few queries cut from a larger
    batch keep that batch's floor).  Returns (ok, stats)."""
    g = np.asarray(g, dtype=np.float64).reshape(-1, 3)
    o = np.asarray(o, dtype=np.float64).reshape(-1, 3)
    kappa = np.asarray(kappa, dtype=np.float64)
    if o.size == 0:
        return True, {"max_rel": 0.0, "mean_rel": 0.0, "ill_conditioned": 0, "n": 0}
    if tau is None:
        tau = float(np.sqrt(np.mean(o * o)))
    tau = max(tau, 1e-30)
    den = np.maximum(np.abs(o), tau)
    relc = np.abs(g - o) / den
    rel = relc.max(axis=1)
    well = kappa <= kappa_well
    rel_gain = np.full_like(o, 0.5) if gain is None else np.asarray(gain, dtype=np.float64).reshape(-1, 3) / den
    boundc = np.where(well[:, None], tol, tol + eps * (1.0 + 2.0 * kappa[:, None]) * rel_gain)
    ok = bool(np.all(relc <= boundc)) and bool(np.all(np.isfinite(g)))
    over = (relc / boundc).max(axis=1)
    bins = {}
    for lo, hi in ((0, 10), (10, 50), (50, 300), (300, 3000), (3000, np.inf)):
        sel = (kappa > lo) & (kappa <= hi)
        if sel.any():
            bins[f"({lo},{hi}]"] = {"n": int(sel.sum()), "max_rel": float(rel[sel].max()),
                                   "max_over_bound": float(over[sel].max())}
    st = {"max_rel": float(rel.max()), "mean_rel": float(rel.mean()),
          "max_rel_well_conditioned": float(rel[well].max()) if well.any() else 0.0,
          "max_rel_ill_conditioned": float(rel[~well].max()) if (~well).any() else 0.0,
          "ill_conditioned": int((~well).sum()), "n": int(len(rel)),
          "worst_over_bound": float(over.max()), "by_kappa": bins}
    return ok, st


def loss(g, y):
    """(L, dL/dg) of the log-space L1 loss over [n,3] outputs."""
    g = np.ascontiguousarray(g, dtype=np.float64)
    y = np.ascontiguousarray(y, dtype=np.float32)
    n = g.shape[0]
    d = np.zeros_like(g)
    val = lib().orc_loss(_ptr(g), _ptr(y), n, _ptr(d))
    return val, d


def albedo_loss(a, t):
    """(L, dL/da) of the albedo head's L2 loss over [n,3] outputs."""
    a = np.ascontiguousarray(a, dtype=np.float64)
    t = np.ascontiguousarray(t, dtype=np.float32)
    n = a.shape[0]
    d = np.zeros_like(a)
    val = lib().orc_albedo_loss(_ptr(a), _ptr(t), n, _ptr(d))
    return val, d


def grad(model: Model, q, dl_dy, with_pyramid=True, with_z=False):
    """Gradients of sum <dl_dy, y> (dl_dy [n, outputs]) w.r.t. frame params, decoder params, pyramid
    and, with_z, the latent of each query ("z", [n][8]: what the encoder of
    Sec. 5.1 back-propagates; with q["z"] given the latents bypass the
    texture and the pyramid gradient stays zero)."""
    if model.frame_form == 1:
        raise NotImplementedError("reverse mode of the paper's frame form is not built")
    n = _nq(q)
    dl = np.ascontiguousarray(dl_dy, dtype=np.float64).reshape(n, model.widths[-1])
    gf = np.zeros(model.n_frame_params(), dtype=np.float64)
    gd = np.zeros(model.n_dec_params(), dtype=np.float64)
    gp = np.zeros((model.texel_count(), 8), dtype=np.float64) if with_pyramid else None
    gz = np.zeros((n, 8), dtype=np.float64) if with_z else None
    qv = _QueryView(q, n)
    lib().orc_grad(C.byref(model._s), C.byref(qv.s), n, _ptr(dl),
                   _ptr(gf) if gf.size else None, _ptr(gd), _ptr(gp), _ptr(gz))
    return {"frame": gf, "decoder": gd, "pyramid": gp, "z": gz}


def split_decoder(model: Model, flat):
    """Split a flat decoder-parameter vector into [(W, b), ...]."""
    out, o = [], 0
    for i in range(len(model.widths) - 1):
        a, b = model.widths[i], model.widths[i + 1]
        W = flat[o:o + a * b].reshape(b, a); o += a * b
        bb = flat[o:o + b]; o += b
        out.append((W, bb))
    return out


def split_frame(model: Model, flat):
    H = model.frame[0][0].shape[0]
    o = 0
    Wf1 = flat[o:o + H * 8].reshape(H, 8); o += H * 8
    bf1 = flat[o:o + H]; o += H
    Wf2 = flat[o:o + 6 * H].reshape(6, H); o += 6 * H
    bf2 = flat[o:o + 6]
    return [(Wf1, bf1), (Wf2, bf2)]


def relative_error(g, o):
    """Max and mean of |g - o| / max(|o|, tau), tau = RMS of o over the batch."""
    g = np.asarray(g, dtype=np.float64)
    o = np.asarray(o, dtype=np.float64)
    if o.size == 0:
        return 0.0, 0.0
    tau = float(np.sqrt(np.mean(o * o)))
    tau = max(tau, 1e-30)
    r = np.abs(g - o) / np.maximum(np.abs(o), tau)
    return float(r.max()), float(r.mean())


# ----------------------------------------------------------------------------
# importance sampling (Sec. 4.3, Appendix A)
# ----------------------------------------------------------------------------
PROXY_FIELDS = ("w_d", "mu_dx", "mu_dy", "w_s", "alpha_x", "alpha_y", "rho", "mu_sx", "mu_sy")


def flat_sampler(layers):
    """[(W [out][in], b), ...] for widths 11-32-32-32-9 -> FP64 flat array."""
    return np.ascontiguousarray(np.concatenate([np.concatenate([W.ravel(), b]) for W, b in layers]),
                                dtype=np.float64)


def qtanh(x):
    return np.array([lib().orc_qtanh(float(v)) for v in np.ravel(x)]).reshape(np.shape(x))


def qsinh(x):
    return np.array([lib().orc_qsinh(float(v)) for v in np.ravel(x)]).reshape(np.shape(x))


def proxy_activate(raw):
    raw = np.ascontiguousarray(raw, dtype=np.float64)
    out = np.zeros(9)
    lib().orc_proxy_activate(_ptr(raw), _ptr(out))
    return out


def proxy_pdf(params, wi, wo):
    """Proxy density of each wo [n][3] given one wi [3]."""
    params = np.ascontiguousarray(params, dtype=np.float64)
    wo = np.ascontiguousarray(np.atleast_2d(wo), dtype=np.float64)
    wi = np.ascontiguousarray(wi, dtype=np.float64)
    out = np.zeros(len(wo))
    lib().orc_proxy_pdf_batch(_ptr(params), _ptr(wi), _ptr(wo), len(wo), _ptr(out))
    return out


def proxy_pdf_h(params, h):
    """Density of specular half vectors at each h [n][3]."""
    params = np.ascontiguousarray(params, dtype=np.float64)
    h = np.ascontiguousarray(np.atleast_2d(h), dtype=np.float64)
    out = np.zeros(len(h))
    lib().orc_proxy_pdf_h_batch(_ptr(params), _ptr(h), len(h), _ptr(out))
    return out


def proxy_sample(params, wi, u):
    """Samples for variates u [n][3]: (wo [n][3], pdf [n])."""
    params = np.ascontiguousarray(params, dtype=np.float64)
    wi = np.ascontiguousarray(wi, dtype=np.float64)
    u = np.ascontiguousarray(u, dtype=np.float64)
    wo = np.zeros((len(u), 3))
    pdf = np.zeros(len(u))
    L = lib()
    for k in range(len(u)):
        L.orc_proxy_sample(_ptr(params), _ptr(wi), _ptr(u[k]), _ptr(wo[k]), _ptr(pdf[k:]))
    return wo, pdf


def sampler_params(model: Model, sampler, q) -> np.ndarray:
    sp = flat_sampler(sampler)
    n = _nq(q)
    out = np.zeros((n, 9))
    qv = _QueryView(q, n)
    lib().orc_sampler_params(C.byref(model._s), _ptr(sp), C.byref(qv.s), n, _ptr(out))
    return out


def sampler_pdf(model: Model, sampler, q) -> np.ndarray:
    sp = flat_sampler(sampler)
    n = _nq(q)
    out = np.zeros(n)
    qv = _QueryView(q, n)
    lib().orc_sampler_pdf(C.byref(model._s), _ptr(sp), C.byref(qv.s), n, _ptr(out))
    return out


def sampler_sample(model: Model, sampler, q, u):
    sp = flat_sampler(sampler)
    n = _nq(q)
    u = np.ascontiguousarray(u, dtype=np.float64)
    wo = np.zeros((n, 3))
    pdf = np.zeros(n)
    qv = _QueryView(q, n)
    lib().orc_sampler_sample(C.byref(model._s), _ptr(sp), C.byref(qv.s), n, _ptr(u), _ptr(wo), _ptr(pdf))
    return wo, pdf


# ----------------------------------------------------------------------------
# encoder (Sec. 5.1): material parameters k(x) -> latent z(x), used in the
# first training phase in place of the latent texture and then evaluated
# once per texel to initialise it
# ----------------------------------------------------------------------------
def encoder_forward(layers, k) -> np.ndarray:
    """z = E(k) for k [n][K]; layers [(W [out][in], b [out]), ...] with ReLU
    hidden layers and a linear output (FP64)."""
    a = np.asarray(k, dtype=np.float64)
    for l, (W, b) in enumerate(layers):
        s = a @ np.asarray(W, dtype=np.float64).T + np.asarray(b, dtype=np.float64)
        a = s if l == len(layers) - 1 else np.maximum(s, 0.0)
    return a


def encoder_grad(layers, k, dz):
    """Gradients of sum_i <dz_i, E(k_i)> with respect to every (W, b), by the
    chain rule through the layers above (ReLU'(0) = 0)."""
    acts, pres = [np.asarray(k, dtype=np.float64)], []
    for l, (W, b) in enumerate(layers):
        s = acts[-1] @ np.asarray(W, dtype=np.float64).T + np.asarray(b, dtype=np.float64)
        pres.append(s)
        acts.append(s if l == len(layers) - 1 else np.maximum(s, 0.0))
    d = np.asarray(dz, dtype=np.float64)
    out = [None] * len(layers)
    for l in range(len(layers) - 1, -1, -1):
        out[l] = (d.T @ acts[l], d.sum(axis=0))
        if l > 0:
            d = (d @ np.asarray(layers[l][0], dtype=np.float64)) * (pres[l - 1] > 0.0)
    return out


def flat_encoder(layers) -> np.ndarray:
    """Per layer W (out x in, row-major) then b: the library's layout."""
    return np.concatenate([np.concatenate([np.asarray(W, np.float64).ravel(), np.asarray(b, np.float64)])
                           for W, b in layers])
