"""torch.autograd bridge to the hand-written CUDA adjoint.

``ensemble_loss(params, handle)`` returns the per-net local objectives
L_{k,m} (Eq. (16)) of every subdomain net as a tensor ``[n_nets]``.  Its
forward runs the grouped kernels without the reverse pass (losses only);
its backward runs them again with the reverse pass - the forward of each
tile is recomputed next to its adjoint instead of being kept alive between
the two calls - and scales each net's gradient by the incoming gradient of
its loss.  Nothing is differentiated by autograd itself: the Jacobian
product is the library's adjoint.

As in Algorithm 1, the neighbour messages a net's ghost terms compare
against are constants of its gradient: d L_{k,m} / d theta_{k,m} only, so
the Jacobian of the vector of losses is block-diagonal and the backward of
``sum(losses)`` is not the total derivative through the messages.

``EnsembleModule`` holds the flat parameter tensor (canonical per-net block
order of ``include/dpinn.h``) so that any torch optimiser can drive it.
"""
from __future__ import annotations

import torch

from .binding import Dpinn


class _EnsembleLoss(torch.autograd.Function):
    @staticmethod
    def forward(ctx, params: torch.Tensor, handle: Dpinn):
        flat = params.detach().contiguous()
        handle.set_params(flat)
        handle.eval_loss()
        rec = handle.loss()
        ctx.handle = handle
        ctx.save_for_backward(params)
        return torch.from_numpy(rec[:, 5].copy()).to(device=params.device, dtype=params.dtype)

    @staticmethod
    def backward(ctx, grad_out: torch.Tensor):
        (params,) = ctx.saved_tensors
        h = ctx.handle
        h.set_params(params.detach().contiguous())
        h.eval_grad()
        g = torch.empty((h.n_nets, h.n_params), device=params.device, dtype=torch.float32)
        h.grad_into(g)
        g = g * grad_out.reshape(-1, 1).to(g.dtype)
        return g.reshape(-1).to(params.dtype), None


def ensemble_loss(params: torch.Tensor, handle: Dpinn) -> torch.Tensor:
    """Per-net losses [n_nets] of the ensemble at ``params`` (differentiable)."""
    if params.numel() != handle.n_nets * handle.n_params:
        raise ValueError(f"params must hold {handle.n_nets * handle.n_params} values")
    if params.dtype != torch.float32:
        raise TypeError("params must be float32")
    return _EnsembleLoss.apply(params, handle)


class EnsembleModule(torch.nn.Module):
    """All subdomain networks as one module with a flat float32 parameter."""

    def __init__(self, handle: Dpinn, params=None):
        super().__init__()
        self.handle = handle
        if params is None:
            params = handle.get_state()[0]
        self.theta = torch.nn.Parameter(torch.as_tensor(params, dtype=torch.float32).reshape(-1).cuda().clone())

    def forward(self) -> torch.Tensor:
        return ensemble_loss(self.theta, self.handle)
