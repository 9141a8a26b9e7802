"""GB300-native batched neural-BRDF evaluation (Zeltner et al., Real-Time
Neural Appearance Models).  The compute lives in libnam.so (CUDA, sm_103a,
C ABI in include/nam.h); this package is its Python binding plus thin
conveniences for building material descriptors from numpy arrays."""
from __future__ import annotations

import ctypes as C

import numpy as np

__all__ = ["B", "Context", "Material", "NamError", "flatten_frame", "flatten_decoder"]


def __getattr__(name):
    # libnam.so is loaded on first use (so that the build step can import
    # this package before the library exists); a missing library raises
    # ImportError there -- there is no fallback.
    import importlib
    if name in ("B", "binding"):
        return importlib.import_module(__name__ + ".binding")
    if name == "NamError":
        return importlib.import_module(__name__ + ".binding").NamError
    raise AttributeError(name)


def flatten_frame(frame):
    """[(Wf1, bf1), (Wf2, bf2)] (frame MLP) or [(Wf, bf)] (the paper's single
    12-output layer) -> FP32 [W, b, ...] (matrices [out][in])."""
    if frame is None:
        return None
    return np.ascontiguousarray(np.concatenate([np.concatenate([W.ravel(), b]) for W, b in frame]),
                                dtype=np.float32)


def flatten_decoder(decoder):
    return np.ascontiguousarray(np.concatenate([np.concatenate([W.ravel(), b]) for W, b in decoder]),
                                dtype=np.float32)


class Context:
    """A libnam context on one GPU."""

    def __init__(self, device=0, hbm_budget_bytes=0, wait_timeout_ns=0, serve_streams=0, serve_queue_depth=0):
        from . import binding as B
        self.device = device
        self.h = B.nam_init(device, hbm_budget_bytes, wait_timeout_ns, serve_streams, serve_queue_depth)

    def close(self):
        from . import binding as B
        if self.h:
            B.nam_shutdown(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def material(self, W0, H0, L, pyramid, frame, decoder, precision=1, filter=0, address=0, trainable=False,
                 act_scale=None, sampler=None, encoder=None):
        """precision: NAM_PREC_F32/F16/FP8 (0/1/2); filter: trilinear/stochastic (0/1); address: wrap/clamp;
        sampler: None or [(W, b)] * 4 of the 11-32-32-32-9 importance-sampling MLP;
        encoder: None or [(W, b)] * 3 of the K-32-32-8 encoder of a trainable material."""
        return Material(self, W0, H0, L, pyramid, frame, decoder, precision, filter, address, trainable, act_scale,
                        sampler, encoder)

    def stats(self):
        from . import binding as B
        return B.nam_get_stats(self.h)

    def check(self):
        from . import binding as B
        B.nam_check_device_error(self.h)


class Material:
    """A neural material resident on the device (pyramid + MLP weights)."""

    def __init__(self, ctx, W0, H0, L, pyramid, frame, decoder, precision, filter, address, trainable, act_scale,
                 sampler=None, encoder=None):
        from . import binding as B
        self.ctx = ctx
        pyr = np.ascontiguousarray(pyramid)
        if pyr.dtype not in (np.float16, np.float32) or pyr.ndim != 2 or pyr.shape[1] != 8:
            raise ValueError("pyramid must be [texels, 8] float16 or float32")
        self._keep = []
        d = B.nam_material_desc()
        d.base_w, d.base_h, d.levels, d.channels = W0, H0, L, 8
        d.latent_dtype = B.NAM_LATENT_F16 if pyr.dtype == np.float16 else B.NAM_LATENT_F32
        d.params_on_device = 0
        d.pyramid = pyr.ctypes.data
        fr = flatten_frame(frame)
        paper = frame is not None and len(frame) == 1
        d.frame_form = B.NAM_FRAME_PAPER if paper else B.NAM_FRAME_MLP
        d.frame_hidden = 0 if (frame is None or paper) else frame[0][0].shape[0]
        d.frame_weights = None if fr is None else fr.ctypes.data
        widths = [decoder[0][0].shape[1]] + [W.shape[0] for W, _ in decoder]
        d.n_layers = len(decoder)
        for i, w in enumerate(widths):
            d.widths[i] = w
        dec = flatten_decoder(decoder)
        d.decoder_weights = dec.ctypes.data
        d.precision, d.filter, d.address, d.trainable = precision, filter, address, int(bool(trainable))
        sc = None
        if act_scale is not None:
            sc = np.ascontiguousarray(act_scale, dtype=np.float32)
            d.fp8_act_scale = sc.ctypes.data
        smp = None
        if sampler is not None:
            smp = flatten_decoder(sampler)
            d.sampler_hidden = sampler[0][0].shape[0]
            d.sampler_weights = smp.ctypes.data
        enc = None
        if encoder is not None:
            enc = flatten_decoder(encoder)
            d.encoder_inputs = encoder[0][0].shape[1]
            d.encoder_weights = enc.ctypes.data
        self._keep = [pyr, fr, dec, sc, smp, enc]
        self.h = B.nam_create_material(ctx.h, d)
        self._keep = []
        self.precision, self.filter, self.address = precision, filter, address
        self.widths = widths
        self.info = B.nam_material_get_info(ctx.h, self.h)

    def destroy(self):
        from . import binding as B
        if self.h:
            B.nam_destroy_material(self.ctx.h, self.h)
            self.h = None

    def eval(self, q, out=None, stream=None, flags=0):
        """q: dict of CUDA float32 tensors (binding.QUERY_FIELDS).  Returns [n, 3]."""
        import torch

        from . import binding as B
        n = int(q["u"].shape[0])
        if out is None:
            out = torch.empty((n, 3), dtype=torch.float32, device=q["u"].device)
        if stream is None:
            stream = torch.cuda.current_stream(q["u"].device)
        B.nam_eval(self.ctx.h, self.h, q, n, out, stream, flags)
        return out

    def eval_albedo(self, q, stream=None, flags=0):
        """(rgb [n, 3], albedo [n, 3]) of a material with the albedo head."""
        import torch

        from . import binding as B
        n = int(q["u"].shape[0])
        rgb = torch.empty((n, 3), dtype=torch.float32, device=q["u"].device)
        alb = torch.empty((n, 3), dtype=torch.float32, device=q["u"].device)
        if stream is None:
            stream = torch.cuda.current_stream(q["u"].device)
        B.nam_eval_albedo(self.ctx.h, self.h, q, n, rgb, alb, stream, flags)
        return rgb, alb

    def eval_host(self, q, out=None, stream=None, flags=0):
        """q: dict of host float32 arrays (numpy or pinned torch).  Synchronous."""
        from . import binding as B
        n = int(q["u"].shape[0])
        if out is None:
            out = np.empty((n, 3), dtype=np.float32)
        B.nam_eval_host(self.ctx.h, self.h, q, n, out, stream, flags)
        return out

    def params(self):
        """(params, pyramid) device pointers of a trainable material."""
        from . import binding as B
        return B.nam_material_params(self.ctx.h, self.h)
