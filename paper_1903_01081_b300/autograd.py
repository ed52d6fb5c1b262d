"""``torch.autograd.Function`` over the discrete adjoint of the time loop.

``emt_loss(params, net, v_target, n_steps)`` returns the loss
J = sum_n ||v_n - v*_n||^2 of ``net`` run with the parameters
``params = [branch values..., source amplitudes...]``; ``backward`` gives
dJ/dparams from the CUDA adjoint (``emt_adjoint``).  One call of
``emt_adjoint`` computes both the loss and the gradient, so the forward
already holds the gradient and the backward only scales it.  ``v_target``
is treated as a constant (it receives no gradient).
"""
from __future__ import annotations

import numpy as np
import torch

from . import emt


class EmtLoss(torch.autograd.Function):
    @staticmethod
    def forward(ctx, params, net, v_target, n_steps, ckpt_every):
        p = params.detach().to("cpu", torch.float64).numpy()
        nb = net.n_branches
        if p.shape != (nb + net.n_sources,):
            raise ValueError(f"params must have {nb + net.n_sources} entries (branch values, then source amplitudes)")
        run = net.copy()
        run.br_value = np.ascontiguousarray(p[:nb])
        run.src_amp = np.ascontiguousarray(p[nb:])
        c = emt.emt_build_network(run)
        try:
            emt.emt_prefactor(c)
            stream = torch.cuda.current_stream() if isinstance(v_target, torch.Tensor) else None
            loss, grad = emt.emt_adjoint(c, v_target, n_steps, ckpt_every, stream=stream)
        finally:
            emt.emt_destroy(c)
        grad = torch.as_tensor(grad).to(params.device)
        ctx.save_for_backward(grad)
        return torch.tensor(loss, dtype=torch.float64, device=params.device)

    @staticmethod
    def backward(ctx, grad_output):
        (grad,) = ctx.saved_tensors
        return grad_output * grad, None, None, None, None


def emt_loss(params: torch.Tensor, net, v_target, n_steps: int, ckpt_every: int = 256) -> torch.Tensor:
    """Differentiable loss of one network run (see module docstring).

    ``v_target``: [n_steps][n_nodes] float64, a numpy array or a CUDA tensor."""
    return EmtLoss.apply(params, net, v_target, int(n_steps), int(ckpt_every))


def parameters_of(net) -> np.ndarray:
    """[branch values..., source amplitudes...] of a network."""
    return np.concatenate([np.asarray(net.br_value, np.float64), np.asarray(net.src_amp, np.float64)])
