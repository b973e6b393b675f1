"""The overlap operator and the U(1) vector-current estimator (test infrastructure).

Overlap Dirac operator at chemical potential mu (Sec. 1, Eq. overlap, lattice
spacing a = 1):

    D_ov = 1 + gamma5 sgn(H(mu)),      H(mu) = gamma5 D_w(mu),

applied to a vector with the k-step TSL approximation of sgn(H) b (``tsl``).
Its adjoint follows from sgn(H)^dagger = sgn(H^dagger) (sgn(lambda) =
sgn(Re lambda) is real) and H(mu)^dagger = H(-mu) (gamma5-hermiticity of Eq.
WD_op):  D_ov^dagger b = b + sgn(H(-mu)) gamma5 b.

U(1) vector current (Sec. 4.3, Eq. lat_vec_cur):

    j_{x,nu} = Tr( D_ov^{-1} dD_ov / dTheta_{x,nu} ),

with the Abelian field Theta entering as U_nu(x) -> e^{i Theta_{x,nu}} U_nu(x)
(App. A, Eq. WD_op with Theta; the backward hop carries the conjugate phase
through U^dagger).  The trace is estimated with Z2 noise vectors eta
(E[eta eta^dagger] = 1): for one eta,

    j_{x,nu}(eta) = eta^dagger D_ov^{-1} (dD_ov/dTheta_{x,nu}) eta
                  = < gamma5 chi, d(sgn(H) eta)/dTheta_{x,nu} >,   chi = D_ov^{-dagger} eta,

because dD_ov/dTheta = gamma5 dsgn(H)/dTheta.  For all links at once this is a
pair of vector-Jacobian products of the TSL map eta -> sgn(H) eta: with the
cotangent xbar = gamma5 chi the VJP gives dL/dU for L = Re <xbar, x>, and with
i xbar the one for Im <xbar, x>.  A link gradient g (dL = Re sum conj(g) dU)
becomes a Theta derivative through dU = i U dTheta:

    dL/dTheta_{x,nu} = Re sum_ab conj(g_ab) i U_ab = -Im sum_ab conj(g_ab) U_ab.

Gauge invariance Theta_{x,nu} -> Theta_{x,nu} + phi_x - phi_{x+nu} makes the
divergence sum_nu (j_{x,nu} - j_{x-nu,nu}) of the exact trace vanish (Sec. 4.3,
Eq. divergence_def); the Z2 estimator reaches it on average.

Exact dense forms (small lattices only) serve as pins: D_ov from the dense H
with the Newton sign of ``ksign``, its log-determinant, and dD_ov/dTheta.
"""
from __future__ import annotations

import numpy as np

from . import dirac, ksign, tsl, vjp

GAMMA5_DIAG = np.array([1.0, 1.0, -1.0, -1.0])


def gamma5(psi):
    """gamma5 psi (chiral basis: diag(1, 1, -1, -1) on the spin index)."""
    return psi * GAMMA5_DIAG[:, None]


def apply_dov(u, b, mu, m_w, k, dagger=False, rebiorth=1, passes=2):
    """D_ov b (or D_ov^dagger b) with the k-step TSL for the sign."""
    b = np.asarray(b, dtype=np.complex128)
    if not dagger:
        return b + gamma5(tsl.tsl_forward(u, b, mu, m_w, k, rebiorth=rebiorth, passes=passes).x)
    return b + tsl.tsl_forward(u, gamma5(b), -mu, m_w, k, rebiorth=rebiorth, passes=passes).x


def theta_derivative(g, u):
    """dL/dTheta per link (shape u.shape[:-2]) from a link gradient g of L."""
    return -np.imag(np.einsum("...ab,...ab->...", np.conj(g), u))


def current_estimate(u, eta, chi, mu, m_w, k, rebiorth=1, passes=2):
    """j_{x,nu}(eta) = < gamma5 chi, d(sgn(H) eta)/dTheta_{x,nu} > for all links,
    complex, shape (Nt, Nz, Ny, Nx, 4): two VJPs of the TSL map on one forward pass."""
    xbar = gamma5(np.asarray(chi, dtype=np.complex128))
    fwd = tsl.tsl_forward(u, eta, mu, m_w, k, rebiorth=rebiorth, passes=passes)
    g_re, _, _ = vjp.tsl_vjp(u, eta, mu, m_w, k, xbar, rebiorth=rebiorth, passes=passes, fwd=fwd)
    g_im, _, _ = vjp.tsl_vjp(u, eta, mu, m_w, k, 1j * xbar, rebiorth=rebiorth, passes=passes, fwd=fwd)
    return theta_derivative(g_re, u) + 1j * theta_derivative(g_im, u)


def divergence(j):
    """sum_nu (j_{x,nu} - j_{x-nu,nu}) per site (Eq. divergence_def), periodic."""
    out = np.zeros(j.shape[:4], dtype=j.dtype)
    for nu in range(4):
        out += j[..., nu] - np.roll(j[..., nu], 1, axis=3 - nu)
    return out


# ---------------------------------------------------------------------------
# exact dense forms (small lattices)
# ---------------------------------------------------------------------------
def dense_h(u, mu, m_w):
    """H(mu) as a dense n x n matrix (n = 12 V), column i = H e_i."""
    shape = u.shape[:4] + (4, 3)
    n = int(np.prod(shape))
    h = np.zeros((n, n), dtype=np.complex128)
    for i in range(n):
        e = np.zeros(n, dtype=np.complex128)
        e[i] = 1.0
        h[:, i] = dirac.apply_h(u, e.reshape(shape), mu, m_w).ravel()
    return h


def dense_dov(u, mu, m_w):
    """Exact D_ov = 1 + gamma5 sgn(H) (dense, Newton sign)."""
    h = dense_h(u, mu, m_w)
    n = h.shape[0]
    g5 = np.tile(np.repeat(GAMMA5_DIAG, 3), n // 12)
    return np.eye(n, dtype=np.complex128) + g5[:, None] * ksign.sign_newton(h)


def with_theta(u, site, nu, theta):
    """Links with the U(1) phase e^{i theta} on the link (site, nu)."""
    out = np.array(u, dtype=np.complex128, copy=True)
    out[site + (nu,)] *= np.exp(1j * theta)
    return out


def exact_current(u, mu, m_w, site, nu, h=1e-5):
    """Tr(D_ov^{-1} dD_ov/dTheta_{site,nu}) with dD_ov/dTheta by central differences
    of the exact dense D_ov."""
    d0 = dense_dov(u, mu, m_w)
    dp = dense_dov(with_theta(u, site, nu, h), mu, m_w)
    dm = dense_dov(with_theta(u, site, nu, -h), mu, m_w)
    return np.trace(np.linalg.solve(d0, (dp - dm) / (2 * h)))


def dlogdet_dtheta(u, mu, m_w, site, nu, h=1e-5):
    """d/dTheta_{site,nu} log det D_ov by central differences of slogdet: the real
    part from log|det|, the imaginary part from the change of the phase of det."""
    sp, lp = np.linalg.slogdet(dense_dov(with_theta(u, site, nu, h), mu, m_w))
    sm, lm = np.linalg.slogdet(dense_dov(with_theta(u, site, nu, -h), mu, m_w))
    return (lp - lm) / (2 * h) + 1j * np.angle(sp / sm) / (2 * h)
