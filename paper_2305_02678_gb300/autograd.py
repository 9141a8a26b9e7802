"""torch.autograd.Function over the neural-BRDF forward (nam_eval) and its
hand-written reverse mode (nam_backward).

The paper fits the latent pyramid, the frame layer and the decoder jointly by
gradient descent on a log-space L1 loss (Sec. 5).  nam_train_step does the
whole step inside the library; this module instead lets torch own the loss
and the optimiser: the material's FP32 parameters and pyramid are exposed as
zero-copy torch tensors (nn.Parameter), the forward runs libnam's FP32
kernel on them, and the backward runs libnam's reverse-mode kernel, which
returns the weight gradients and scatters the latent gradients into the
pyramid-shaped gradient with atomics.  Every step of the evaluation and of
its derivative runs in libnam; torch only holds memory and runs the loss and
the optimiser update.
"""
from __future__ import annotations

import torch

from . import binding as B

__all__ = ["NeuralBRDFFunction", "NeuralMaterial", "material_tensors", "log_l1_loss"]


class _DevArray:
    """CUDA array interface over a libnam-owned FP32 device buffer."""

    def __init__(self, ptr, n):
        self.__cuda_array_interface__ = {"shape": (int(n),), "typestr": "<f4", "data": (int(ptr), False),
                                         "version": 3}


def material_tensors(mat):
    """Zero-copy torch views of a trainable material's parameters: the MLP
    weights and biases ([n_params], frame layers first, then the decoder, each
    layer W row-major [out][in] followed by b) and the latent pyramid
    ([texels, 8], levels finest first).  The views alias libnam's storage: the
    material must outlive them, and writes to them change what nam_eval reads."""
    p, z = mat.params()
    dev = torch.device("cuda", mat.ctx.device)
    params = torch.as_tensor(_DevArray(p, mat.info.n_params), device=dev)
    pyramid = torch.as_tensor(_DevArray(z, mat.info.texels * 8), device=dev).view(mat.info.texels, 8)
    return params, pyramid


class NeuralBRDFFunction(torch.autograd.Function):
    """rgb = g(z(uv, lod), T wi, T wo) for a batch of queries (Eq. 3 with the
    frame of Sec. 4.1), differentiable in the material's parameters and
    latent pyramid.  `params` and `pyramid` must be the tensors
    material_tensors() returned for `mat`: the kernels read the material's own
    storage, and the tensors are passed so that autograd routes gradients to
    them (and notices in-place updates between forward and backward).  With
    the albedo head (six decoder outputs) the result is [n, 6]: RGB, then the
    directional albedo, and the gradient flowing back has that layout."""

    @staticmethod
    def forward(ctx, params, pyramid, mat, queries, flags):
        p, z = mat.params()
        if params.data_ptr() != p or pyramid.data_ptr() != z:
            raise ValueError("params/pyramid must be the material's own tensors (material_tensors)")
        n = int(queries["u"].shape[0])
        stream = torch.cuda.current_stream(params.device)
        if mat.widths[-1] == 6:
            rgb = torch.empty((n, 3), dtype=torch.float32, device=params.device)
            alb = torch.empty((n, 3), dtype=torch.float32, device=params.device)
            B.nam_eval_albedo(mat.ctx.h, mat.h, queries, n, rgb, alb, stream, flags)
            out = torch.cat([rgb, alb], dim=1)
        else:
            out = torch.empty((n, 3), dtype=torch.float32, device=params.device)
            B.nam_eval(mat.ctx.h, mat.h, queries, n, out, stream, flags)
        ctx.save_for_backward(params, pyramid)
        ctx.mat, ctx.queries, ctx.flags, ctx.n = mat, queries, flags, n
        return out

    @staticmethod
    def backward(ctx, grad_rgb):
        params, pyramid = ctx.saved_tensors
        mat = ctx.mat
        gp = torch.zeros_like(params) if ctx.needs_input_grad[0] else None
        gz = torch.zeros_like(pyramid) if ctx.needs_input_grad[1] else None
        if grad_rgb.shape != (ctx.n, mat.widths[-1]):
            raise ValueError(f"output gradient of shape {tuple(grad_rgb.shape)}, expected ({ctx.n}, {mat.widths[-1]})")
        if gp is not None or gz is not None:
            B.nam_backward(mat.ctx.h, mat.h, ctx.queries, ctx.n, grad_rgb.contiguous().float(), gp, gz,
                           torch.cuda.current_stream(params.device), ctx.flags)
        return gp, gz, None, None, None


class NeuralMaterial(torch.nn.Module):
    """A trainable neural material (FP32 parameters and FP32 latents) whose
    parameters are nn.Parameters over libnam's storage, for use with torch
    losses and optimisers."""

    def __init__(self, context, W0, H0, L, pyramid, frame, decoder, filter=0, address=0):
        super().__init__()
        self.material = context.material(W0, H0, L, pyramid, frame, decoder, precision=B.NAM_PREC_F32,
                                         filter=filter, address=address, trainable=True)
        p, z = material_tensors(self.material)
        self.params = torch.nn.Parameter(p)
        self.pyramid = torch.nn.Parameter(z)

    def forward(self, queries, cosine=False):
        return NeuralBRDFFunction.apply(self.params, self.pyramid, self.material, queries,
                                        B.NAM_OUT_COSINE if cosine else 0)


def log_l1_loss(rgb, target):
    """Mean over the batch and channels of |log(1 + max(g, 0)) - log(1 + y)|
    plus 0.01 * max(-g, 0): the paper's L1 loss in log space (Sec. 5), with a
    small linear penalty so that negative outputs still receive a gradient."""
    d = torch.log1p(torch.relu(rgb)) - torch.log1p(target)
    return (d.abs() + 0.01 * torch.relu(-rgb)).mean()
