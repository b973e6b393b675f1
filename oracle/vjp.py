"""Reverse-mode derivative (VJP) of the TSL map b -> x with respect to all links and mu.

Loss convention: L = Re <xbar, x> = Re sum conj(xbar_i) x_i.  Gradients of complex
quantities z are "conjugate-Wirtinger" vectors g_z with dL = Re <g_z, dz>, so
that the returned dU matches the convention of torch autograd for complex
leaves (all 9 entries of each link treated as independent).

The derivative generalises App. A, Eq. dWD_op from the U(1) phase Theta to
every SU(3) link entry and to mu, and runs the TSL recurrence of ``tsl`` in
reverse.  Primitive rules used (z = a u; c = u^dagger w; ...):

    z = a u          : g_u += conj(a) g_z,      g_a += u^dagger g_z
    c = u^dagger w   : g_w += u g_c,            g_u += w conj(g_c)
    delta = sqrt|w|  : g_w += g_delta w / (2 delta |w|)      (delta real)
    beta = w / delta : g_w += g_beta / delta,   g_delta -= Re(conj(w) g_beta) / delta^2
    w' = s / conj(b) : g_s += g_w' / b,         g_b -= conj(s^dagger g_w') / conj(b)^2
    p = H v          : g_v += H^dagger g_p,     g_H += g_p v^dagger
    q = H^dagger w   : g_w += H g_q,            g_H += w g_q^dagger
    y = beta_0 sgn(T) e_1 : G_T = L_sgn(T^dagger, beta_0 g_y e_1^T)    (Theorem 1)

Re-biorthogonalisation is differentiated like every other step.  One
classical Gram-Schmidt pass r' = r - V c, c = W^dagger r  (and s' = s - W d,
d = V^dagger s) has the adjoint

    e_r = V^dagger g_r',  e_s = W^dagger g_s'
    g_r = g_r' - W e_r,   g_s = g_s' - V e_s
    g_{v_i} += -g_r' conj(c_i) - s conj(e_s,i),   g_{w_i} += -r conj(e_r,i) - g_s' conj(d_i)

In exact arithmetic these terms cancel (W^dagger r vanishes identically), but
in floating point they are what keeps the reverse sweep stable: without them
the adjoint of the recurrence grows without bound once k is a few hundred.
The pre-pass vectors are rebuilt from the stored basis and coefficients,
r_in = r_out + V c, starting from r = delta_{j+1} v_{j+1}.

The contraction of g_H = sum a b^dagger into (dU, dmu) is ``dirac.link_gradient``.

``emulate_fp32`` estimates how far an implementation that keeps its lattice
vectors in FP32 can be from the FP64 result: as in ``tsl.tsl_forward``, the
links and every stored or produced lattice vector (here also every cotangent
vector of the reverse sweep) are rounded to complex64, while the dots, the
recurrence scalars, the k x k sign and its Frechet adjoint, and the final
contraction stay in FP64.
"""
from __future__ import annotations

import numpy as np

from . import dirac, ksign, tsl as tslmod


def tsl_vjp(u, b, mu, m_w, k, xbar, rebiorth=1, passes=2, fwd=None, emulate_fp32=False):
    """Return (dU, dmu, fwd) for L = Re <xbar, TSL_k(H(U, mu)) b>."""
    if fwd is None:
        fwd = tslmod.tsl_forward(u, b, mu, m_w, k, rebiorth=rebiorth, passes=passes, emulate_fp32=emulate_fp32)
    v, w = fwd.v, fwd.w
    alpha, beta, delta, y = fwd.alpha, fwd.beta, fwd.delta, fwd.y
    xbar = np.asarray(xbar, dtype=np.complex128)
    rnd = tslmod._round32 if emulate_fp32 else tslmod._identity
    uu = rnd(np.asarray(u, dtype=np.complex128))

    def h(psi):
        return rnd(dirac.apply_h(uu, psi, mu, m_w))

    def hdag(psi):
        return rnd(dirac.apply_h_dagger(uu, psi, mu, m_w))

    # g_y = V^dagger xbar;  G_F = beta_0 g_y e_1^T;  G_T = L_sgn(T^dagger, G_F)
    g_y = np.array([np.vdot(v[j], xbar) for j in range(k)])
    g_f = np.zeros((k, k), dtype=np.complex128)
    g_f[:, 0] = fwd.beta0 * g_y
    g_t = ksign.frechet_adjoint_sign(fwd.t, g_f)
    g_alpha_t = np.diag(g_t).copy()
    g_beta_t = np.zeros(k, dtype=np.complex128)
    g_delta_t = np.zeros(k, dtype=np.float64)
    for j in range(1, k):
        g_beta_t[j] = g_t[j - 1, j]
        g_delta_t[j] = np.real(g_t[j, j - 1])

    terms_a, terms_b = [], []
    vm_all = np.stack([a.ravel() for a in v], axis=1)
    wm_all = np.stack([a.ravel() for a in w], axis=1)
    acc_v = np.zeros((k,) + xbar.shape, dtype=np.complex128)   # projection-adjoint terms
    acc_w = np.zeros((k,) + xbar.shape, dtype=np.complex128)

    # last index (0-based k-1): only alpha_k = w_k^dagger H v_k
    j = k - 1
    g_a = g_alpha_t[j]
    g_p = rnd(w[j] * g_a)
    gv = rnd(np.conj(y[j]) * xbar + hdag(g_p))     # complete gradient of v[k-1]
    gw = rnd(h(v[j]) * np.conj(g_a))               # complete gradient of w[k-1]
    terms_a.append(g_p)
    terms_b.append(v[j])

    pv = np.zeros_like(xbar)     # partial gradient of v[j] carried from step j+1
    pw = np.zeros_like(xbar)
    carry_beta = 0.0 + 0.0j      # gradient of beta[j+1] from step j+1's r
    carry_delta = 0.0            # gradient of delta[j+1] from step j+1's s
    for j in range(k - 2, -1, -1):
        d = delta[j + 1]
        bt = beta[j + 1]
        omega = bt * d
        # v[j+1] = r / d,  w[j+1] = s / conj(bt)
        g_d = g_delta_t[j + 1] + carry_delta - np.real(np.vdot(v[j + 1], gv)) / d
        g_b = g_beta_t[j + 1] + carry_beta - np.conj(np.vdot(w[j + 1], gw)) / np.conj(bt)
        g_r = gv / d
        g_s = gw / bt
        # bt = omega / d, d = sqrt|omega|
        g_w = g_b / d
        g_d = g_d - np.real(np.conj(omega) * g_b) / d ** 2
        g_w = g_w + g_d * omega / (2.0 * d * abs(omega))
        # omega = s^dagger r with r = d v[j+1], s = conj(bt) w[j+1]
        r_out = d * v[j + 1]
        s_out = np.conj(bt) * w[j + 1]
        g_r = rnd(g_r + s_out * g_w)
        g_s = rnd(g_s + r_out * np.conj(g_w))
        # Gram-Schmidt passes of this step, last pass first
        if j in fwd.proj:
            vm, wm = vm_all[:, :j + 1], wm_all[:, :j + 1]
            for (c, dd) in reversed(fwd.proj[j]):
                r_in = r_out + (vm @ c).reshape(r_out.shape)
                s_in = s_out + (wm @ dd).reshape(s_out.shape)
                e_r = vm.conj().T @ g_r.ravel()
                e_s = wm.conj().T @ g_s.ravel()
                for i in range(j + 1):
                    acc_v[i] -= g_r * np.conj(c[i]) + s_in * np.conj(e_s[i])
                    acc_w[i] -= r_in * np.conj(e_r[i]) + g_s * np.conj(dd[i])
                g_r = rnd(g_r - (wm @ e_r).reshape(g_r.shape))
                g_s = rnd(g_s - (vm @ e_s).reshape(g_s.shape))
                r_out, s_out = r_in, s_in
        # r = p - alpha v[j] - beta[j] v[j-1];  s = q - conj(alpha) w[j] - delta[j] w[j-1]
        g_p = g_r.copy()
        g_q = g_s
        g_a = g_alpha_t[j] - np.vdot(v[j], g_r) - np.conj(np.vdot(w[j], g_s))
        pv = pv - np.conj(alpha[j]) * g_r
        pw = pw - alpha[j] * g_s
        if j > 0:
            new_pv = -np.conj(beta[j]) * g_r
            new_pw = -delta[j] * g_s
            new_carry_beta = -np.vdot(v[j - 1], g_r)
            new_carry_delta = -np.real(np.vdot(w[j - 1], g_s))
        # alpha = w[j]^dagger p
        g_p = rnd(g_p + w[j] * g_a)
        pw = pw + h(v[j]) * np.conj(g_a)
        # p = H v[j], q = H^dagger w[j]; plus the projection terms of later steps
        gv = rnd(pv + np.conj(y[j]) * xbar + hdag(g_p) + acc_v[j])
        gw = rnd(pw + h(g_q) + acc_w[j])
        terms_a += [g_p, w[j]]
        terms_b += [v[j], g_q]
        if j > 0:
            pv, pw = new_pv, new_pw
            carry_beta, carry_delta = new_carry_beta, new_carry_delta

    du, dmu = dirac.link_gradient(np.stack(terms_a), np.stack(terms_b), uu, mu, m_w)
    return du, dmu, fwd
