"""torch.autograd wrappers of F(q, tau) and S(q, w) as functions of
theta = (T, eta, A, B, C) (temperature, broadening, f_xc-model parameters).

Forward: lrtddft_set_params, chi0_assemble, dyson_solve, then itcf_laplace (FOLD form) or dsf.
Backward: lrtddft_itcf_vjp / lrtddft_dsf_vjp, the library's hand-written adjoint (recomputed
Dyson LU from the stored chi0, projections of the pair densities on the GPU).  Argument
marshalling only; every step runs in the CUDA library.

theta is a float64 tensor of shape [5]; the results are float64 tensors [nq][ntau] and
[nq][nw] on theta's device.  One library context serves one graph at a time: when another
forward has changed the context since, backward first restores the state of its own forward.
"""
from __future__ import annotations

import numpy as np
import torch

from . import binding


def _params(theta) -> tuple:
    t = [float(x) for x in theta.detach().cpu().tolist()]
    if len(t) != 5:
        raise ValueError("theta must hold (T, eta, A, B, C)")
    return tuple(t)


def _run(lrt: binding.Context, p: tuple) -> None:
    lrt.set_params(p[0], p[1], fxc_params=p[2:])
    lrt.chi0_assemble()
    lrt.dyson_solve()


def _restore(lrt: binding.Context, p: tuple) -> None:
    cur = (lrt.wl.T, lrt.wl.eta) + tuple(float(x) for x in lrt.wl.fxc_params)
    if cur != p:
        _run(lrt, p)


class ITCF(torch.autograd.Function):
    @staticmethod
    def forward(ctx, theta, lrt, tau):
        p = _params(theta)
        _run(lrt, p)
        tau = np.ascontiguousarray(tau, dtype=np.float64)
        F, _ = lrt.itcf(tau)
        ctx.lrt, ctx.tau, ctx.p = lrt, tau, p
        return torch.from_numpy(F).to(theta.device)

    @staticmethod
    def backward(ctx, gF):
        _restore(ctx.lrt, ctx.p)
        g = ctx.lrt.itcf_vjp(ctx.tau, gF.detach().double().cpu().numpy())
        return torch.from_numpy(g).to(gF.device), None, None


class DSF(torch.autograd.Function):
    @staticmethod
    def forward(ctx, theta, lrt):
        p = _params(theta)
        _run(lrt, p)
        S = lrt.dsf()
        ctx.lrt, ctx.p = lrt, p
        return torch.from_numpy(S).to(theta.device)

    @staticmethod
    def backward(ctx, gS):
        _restore(ctx.lrt, ctx.p)
        g = ctx.lrt.dsf_vjp(gS.detach().double().cpu().numpy())
        return torch.from_numpy(g).to(gS.device), None


def itcf(theta: torch.Tensor, lrt: binding.Context, tau) -> torch.Tensor:
    """F(q, tau) [nq][ntau] (absolute tau, FOLD form), differentiable in theta."""
    return ITCF.apply(theta, lrt, tau)


def dsf(theta: torch.Tensor, lrt: binding.Context) -> torch.Tensor:
    """S(q, w) [nq][nw], differentiable in theta."""
    return DSF.apply(theta, lrt)
