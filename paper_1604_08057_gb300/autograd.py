"""torch.autograd.Function for x = TSL_k(H(U, mu)) b with the library's hand-written VJP.

Forward calls ``ov_tsl_sign_fwd``, which keeps the forward state on the device
(a tape); backward calls ``ov_tsl_sign_vjp_tape`` on it, so the recurrence and
the k x k sign are not recomputed, and returns the conjugate-Wirtinger gradient
of the links (torch's convention for complex leaves) and d/dmu.  The tape is
freed after the backward pass.  The source b is treated as a constant.
"""
from __future__ import annotations

import torch

from . import binding


class OvTSLSign(torch.autograd.Function):
    @staticmethod
    def forward(ctx, u, mu, b, k, m_w=-2.0, precision="fp64", rebiorth=1, passes=2):
        mu_f = float(mu)
        x, tape = binding.tsl_sign_fwd(u, mu_f, m_w, b, k, precision, rebiorth, passes)
        ctx.tape = tape
        ctx.mu_is_tensor = torch.is_tensor(mu)
        ctx.device = u.device
        return x

    @staticmethod
    def backward(ctx, xbar):
        du, dmu = ctx.tape.vjp(xbar.contiguous())
        ctx.tape.free()
        gmu = torch.tensor(dmu, dtype=torch.float64, device=ctx.device) if ctx.mu_is_tensor else None
        return du, gmu, None, None, None, None, None, None


def tsl_sign(u, mu, b, k, m_w=-2.0, precision="fp64", rebiorth=1, passes=2):
    return OvTSLSign.apply(u, mu, b, k, m_w, precision, rebiorth, passes)
