"""torch.autograd bridge to the library's hand-written adjoint.

``visibility_logits(cache, params, pos)`` gives the network's output logits
(one per light, or per cluster) at positions ``pos`` as a differentiable
function of the flat parameter vector ``params`` (hash tables, then the
weight matrices, the layout of ``nvc_synth.param_layout``).  The forward is
the library's encode + MLP (``nvc_mlp_forward``), the backward its adjoint
kernels: the MLP backward and the hash-grid scatter (``nvc_mlp_backward``).
Positions get no gradient.

The cache handle is the compute engine: the forward loads ``params`` into it
(``nvc_set_params``, which leaves its Adam state alone) and the handle keeps
the activations for the backward.  If another forward ran on the same
handle in between, the backward recomputes them first, so any order of
forward and backward calls gives the right gradient.  At most
``batch_positions`` positions per call.
"""
from __future__ import annotations

import torch

from . import nvc as _nvc


class VisibilityLogits(torch.autograd.Function):
    @staticmethod
    def forward(ctx, params, pos, cache):
        params = params.detach().contiguous()
        pos = pos.detach().contiguous()
        _nvc.nvc_set_params(cache.handle, params)
        logits = torch.empty((pos.shape[0], cache.L), device=pos.device, dtype=torch.float32)
        _nvc.nvc_mlp_forward(cache.handle, pos, logits)
        cache._autograd_token = getattr(cache, "_autograd_token", 0) + 1
        ctx.token = cache._autograd_token
        ctx.cache = cache
        ctx.save_for_backward(params, pos)
        return logits

    @staticmethod
    def backward(ctx, dlogits):
        params, pos = ctx.saved_tensors
        cache = ctx.cache
        if getattr(cache, "_autograd_token", None) != ctx.token:
            # the handle's activations belong to a later forward: recompute ours
            _nvc.nvc_set_params(cache.handle, params)
            scratch = torch.empty((pos.shape[0], cache.L), device=pos.device, dtype=torch.float32)
            _nvc.nvc_mlp_forward(cache.handle, pos, scratch)
            cache._autograd_token = ctx.token
        grad = torch.empty(cache.n_params, device=pos.device, dtype=torch.float32)
        _nvc.nvc_mlp_backward(cache.handle, pos, dlogits.detach().float().contiguous(), grad)
        return grad, None, None


def visibility_logits(cache, params: torch.Tensor, pos: torch.Tensor) -> torch.Tensor:
    """Differentiable logits [n, L] of the cache's network at pos [n, 3]."""
    return VisibilityLogits.apply(params, pos, cache)
