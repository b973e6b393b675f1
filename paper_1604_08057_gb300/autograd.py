"""torch.autograd.Function for x = TSL_k(H(U, mu)) b with the library's hand-written VJP.

Forward calls ``ov_tsl_sign``; backward calls ``ov_tsl_sign_vjp`` (which
re-runs the recurrence on the device) and returns the conjugate-Wirtinger
gradient of the links (torch's convention for complex leaves) and d/dmu.
The source b is treated as a constant.
"""
from __future__ import annotations

import torch

from . import binding


class OvTSLSign(torch.autograd.Function):
    @staticmethod
    def forward(ctx, u, mu, b, k, m_w=-2.0, precision="fp64", rebiorth=1, passes=2):
        mu_f = float(mu)
        x = binding.tsl_sign(u, mu_f, m_w, b, k, precision, rebiorth, passes)
        ctx.save_for_backward(u, b)
        ctx.cfg = (mu_f, k, m_w, precision, rebiorth, passes, torch.is_tensor(mu))
        return x

    @staticmethod
    def backward(ctx, xbar):
        u, b = ctx.saved_tensors
        mu, k, m_w, precision, rebiorth, passes, mu_is_tensor = ctx.cfg
        du, dmu, _ = binding.tsl_sign_vjp(u, mu, m_w, b, k, xbar.contiguous(), precision, rebiorth, passes,
                                          want_x=False)
        gmu = torch.tensor(dmu, dtype=torch.float64, device=u.device) if mu_is_tensor else None
        return du, gmu, None, None, None, None, None, None


def tsl_sign(u, mu, b, k, m_w=-2.0, precision="fp64", rebiorth=1, passes=2):
    return OvTSLSign.apply(u, mu, b, k, m_w, precision, rebiorth, passes)
