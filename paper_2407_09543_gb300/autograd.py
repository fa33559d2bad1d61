"""The network as a differentiable torch function over the library's forward and
hand-written backward (ntbc_vjp): argument marshalling only, every step runs in the
CUDA kernels of libntbc."""
from __future__ import annotations

import torch

from ._abi import Model


class NTBCFunction(torch.autograd.Function):
    """(e_hat, c_hat) = NTBCFunction.apply(params, model, block_ids, qat_bits)

    params     device float32 [layout.total]: FP32 master parameters (grids then MLPs in
               the layout of include/ntbc.h), copied into `model` before each pass
    model      a Model of the matching description
    block_ids  device int32 [n]
    qat_bits   0, or 8 / 4: the grids pass through the QAT fake quantiser (Sec. 3.3),
               whose backward is the straight-through mask
    Returns e_hat [n, out_endpoint] and c_hat [n, 16, out_color] (sigmoid outputs). The
    backward recomputes the activations from the parameters (nothing is stored between
    the two passes) and returns d/d params through the library's backward kernels."""

    @staticmethod
    def forward(ctx, params, model: Model, block_ids, qat_bits=0):
        lay = model.layout
        n = block_ids.numel()
        model.set_params(params.detach().contiguous())
        e_hat = torch.empty(n, lay.out_endpoint, device=params.device, dtype=torch.float32)
        c_hat = torch.empty(n, 16, lay.out_color, device=params.device, dtype=torch.float32)
        model.vjp(block_ids, qat_bits, e_hat=e_hat, c_hat=c_hat)
        ctx.model = model
        ctx.qat_bits = qat_bits
        ctx.save_for_backward(params, block_ids)
        return e_hat, c_hat

    @staticmethod
    def backward(ctx, g_e, g_c):
        params, block_ids = ctx.saved_tensors
        model = ctx.model
        lay = model.layout
        n = block_ids.numel()
        if g_e is None:
            g_e = torch.zeros(n, lay.out_endpoint, device=params.device, dtype=torch.float32)
        if g_c is None:
            g_c = torch.zeros(n, 16, lay.out_color, device=params.device, dtype=torch.float32)
        model.set_params(params.detach().contiguous())
        grads = torch.empty_like(params)
        model.vjp(block_ids, ctx.qat_bits, g_e=g_e.float().contiguous(), g_c=g_c.float().contiguous(), grads=grads)
        return grads, None, None, None


def ntbc_apply(params, model: Model, block_ids, qat_bits=0):
    return NTBCFunction.apply(params, model, block_ids, qat_bits)
