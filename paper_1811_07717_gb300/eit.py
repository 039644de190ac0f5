"""Linearised EIT (App. A.3) as a differentiable torch function.

The unknown is the log of a per-element conductivity scale s_m: element m's
tensor is exp(log_s[m]) times its base tensor.  forward() assembles the system
at that conductivity, solves the transfer matrix and returns the electrode
voltages y (np x L, average-referenced) for the current patterns I; backward()
returns dL/dlog_s through the adjoint kernel of libzi:

    dL/dlog_s_m = sum_{p,k} (dL/dy)_{p,k} * (-u_p^T K_m w_k),

contracted per tetrahedron without forming the Jacobian.  The full Jacobian
(m x np x L) is available from eit_jacobian().

Both directions run in libzi; this module only marshals tensors.
"""
from __future__ import annotations

import torch

from . import zi


class EITVoltages(torch.autograd.Function):
    """y = EITVoltages.apply(log_s, system, sigma_base6, I, opts)."""

    @staticmethod
    def forward(ctx, log_s, system, sigma_base6, I, opts):
        system.set_log_conductivity(sigma_base6, log_s.detach())
        system.transfer(opts, want_T=False)
        y, _ = system.eit(I, mode=None, opts=opts)
        ctx.system = system
        ctx.I = I
        ctx.opts = opts
        ctx.version = system.version
        return y

    @staticmethod
    def backward(ctx, grad_y):
        system = ctx.system
        if system.version != ctx.version:
            raise RuntimeError("the system was re-assembled after this forward; "
                               "its transfer matrix no longer matches the saved conductivity")
        _, g = system.eit(ctx.I, mode=zi.EIT_VJP, grad_y=grad_y.contiguous().to(torch.float64),
                          opts=ctx.opts, want_y=False)
        return g, None, None, None, None


def eit_voltages(log_s, system, sigma_base6, I, opts=None):
    """Differentiable electrode voltages y(log_s) (np x L)."""
    return EITVoltages.apply(log_s, system, sigma_base6, I, opts or zi.SolverOpts(tol=1e-12))


def eit_jacobian(system, I, opts=None):
    """Full Jacobian dy_{p,k}/dlog s_m at the system's current conductivity,
    as an (m, np, L) CUDA tensor, plus y."""
    y, J = system.eit(I, mode=zi.EIT_FULL, opts=opts or zi.SolverOpts(tol=1e-12))
    return J, y
