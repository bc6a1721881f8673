"""torch.autograd.Function over the adjoint kernels.

``heston_price(theta, contract, n_paths, n_steps, seed)`` returns the
Monte Carlo price (a 0-dim float64 CUDA tensor) of one contract for the
parameter vector theta = (S0, v0, kappa, theta, xi, rho, r); its backward
runs the hand-written reverse-mode kernel (heston_mc_adjoint_backward), which
rebuilds each path from checkpoints instead of storing it.  The gradient is
the pathwise estimate on the same paths as the price.  Argument marshalling
only: the work is in the CUDA library.
"""
from __future__ import annotations

import torch

from . import native

PARAM_NAMES = ("S0", "v0", "kappa", "theta", "xi", "rho", "r")


class HestonPrice(torch.autograd.Function):
    @staticmethod
    def forward(ctx, theta, contract, n_paths, n_steps, seed):
        vals = [float(x) for x in theta.detach().cpu().tolist()]
        params = native.make_params(*vals)
        dev = torch.device("cuda", torch.cuda.current_device())
        ws_bytes = native.heston_adjoint_workspace_bytes(n_paths, n_steps)
        ws = torch.empty(ws_bytes // 8 + 32, dtype=torch.float64, device=dev)
        out = torch.empty(2, dtype=torch.float64, device=dev)
        opts = native.make_options(prec=native.HESTON_FP32, stream=torch.cuda.current_stream())
        native.heston_mc_adjoint_forward(params, contract, n_paths, n_steps, seed, opts, ws,
                                         ws_bytes, out)
        ctx.save_for_backward(ws)
        ctx.meta = (params, contract, n_paths, n_steps, seed, ws_bytes, theta.device, theta.dtype)
        ctx.price_se = out[1]
        return out[0]

    @staticmethod
    def backward(ctx, grad_out):
        (ws,) = ctx.saved_tensors
        params, contract, n_paths, n_steps, seed, ws_bytes, tdev, tdtype = ctx.meta
        g = torch.empty(14, dtype=torch.float64, device=ws.device)
        opts = native.make_options(prec=native.HESTON_FP32, stream=torch.cuda.current_stream())
        native.heston_mc_adjoint_backward(params, contract, n_paths, n_steps, seed, opts, ws,
                                          ws_bytes, g)
        grad = (grad_out * g[:7]).to(device=tdev, dtype=tdtype)
        return grad, None, None, None, None


def heston_price(theta, contract, n_paths: int, n_steps: int, seed: int):
    """Differentiable price; theta = tensor (S0, v0, kappa, theta, xi, rho, r)."""
    return HestonPrice.apply(theta, contract, n_paths, n_steps, seed)


def price_and_gradient(params: dict, contract, n_paths, n_steps, seed):
    """(price, se), (gradient[7], se[7]) as numpy arrays through the two kernels."""
    theta = torch.tensor([params[k] for k in PARAM_NAMES], dtype=torch.float64, requires_grad=True)
    price = heston_price(theta, contract, n_paths, n_steps, seed)
    dev = price.device
    p = native.make_params(*[params[k] for k in PARAM_NAMES])
    ws_bytes = native.heston_adjoint_workspace_bytes(n_paths, n_steps)
    ws = torch.empty(ws_bytes // 8 + 32, dtype=torch.float64, device=dev)
    out = torch.empty(2, dtype=torch.float64, device=dev)
    g = torch.empty(14, dtype=torch.float64, device=dev)
    opts = native.make_options(prec=native.HESTON_FP32, stream=torch.cuda.current_stream())
    native.heston_mc_adjoint_forward(p, contract, n_paths, n_steps, seed, opts, ws, ws_bytes, out)
    native.heston_mc_adjoint_backward(p, contract, n_paths, n_steps, seed, opts, ws, ws_bytes, g)
    torch.cuda.synchronize()
    return out.cpu().numpy(), (g[:7].cpu().numpy(), g[7:].cpu().numpy())
