"""Wilson-Dirac operator at chemical potential mu (App. A, Eqs. WD_op, WD_G).

    D_w(mu) = 1 - kappa sum_{i=1..3} (G_i^+ + G_i^-) - kappa (e^{mu} G_4^+ + e^{-mu} G_4^-)
    (G_nu^+)_{x,y} = (1 + gamma_nu) U_nu(x)            delta_{x+nu, y}
    (G_nu^-)_{x,y} = (1 - gamma_nu) U_nu(x - nu)^dag   delta_{x-nu, y}
    kappa = 1 / (2 m_W + 8),    H(mu) = gamma5 D_w(mu)   (Sec. 1, Eq. overlap)

Readings where App. A is silent:
* U_{-nu}(x) = U_nu(x - nu)^dagger (needed for gamma5-hermiticity).
* Theta = 0 (no background U(1) field): it can be folded into U.
* periodic boundary conditions in all four directions.
* Euclidean chiral gamma basis:  gamma_k = [[0, -i sigma_k], [i sigma_k, 0]],
  gamma_4 = [[0, 1], [1, 0]],  gamma5 = gamma_1 gamma_2 gamma_3 gamma_4.

Array layout: spinors (..., Nt, Nz, Ny, Nx, 4, 3); links (Nt, Nz, Ny, Nx, 4, 3, 3)
with direction index 0..3 = x, y, z, t.  All arithmetic is complex128.
"""
from __future__ import annotations

import numpy as np

_S1 = np.array([[0, 1], [1, 0]], dtype=np.complex128)
_S2 = np.array([[0, -1j], [1j, 0]], dtype=np.complex128)
_S3 = np.array([[1, 0], [0, -1]], dtype=np.complex128)
_Z2 = np.zeros((2, 2), dtype=np.complex128)
_I2 = np.eye(2, dtype=np.complex128)

GAMMA = [np.block([[_Z2, -1j * s], [1j * s, _Z2]]) for s in (_S1, _S2, _S3)]
GAMMA.append(np.block([[_Z2, _I2], [_I2, _Z2]]))
GAMMA5 = GAMMA[0] @ GAMMA[1] @ GAMMA[2] @ GAMMA[3]
ID4 = np.eye(4, dtype=np.complex128)


def kappa_of(m_w: float) -> float:
    """Hopping parameter kappa = 1/(2 m_W + 8) (App. A)."""
    return 1.0 / (2.0 * m_w + 8.0)


def hop_factor(nu: int, mu: float) -> float:
    """e^{mu} on the forward temporal hop (nu = t), 1 otherwise (Eq. WD_op)."""
    return float(np.exp(mu)) if nu == 3 else 1.0


def shift(field: np.ndarray, nu: int, sign: int) -> np.ndarray:
    """field(x + sign * nu_hat) with periodic wrap.

    Works for spinors (..., 4, 3) and single-direction links (..., 3, 3): the
    lattice axis of direction nu is the (3 + nu)-th axis from the end.
    """
    return np.roll(field, -sign, axis=-3 - nu)


def spin_mul(m: np.ndarray, psi: np.ndarray) -> np.ndarray:
    return np.einsum("st,...tc->...sc", m, psi)


def colour_mul(u: np.ndarray, psi: np.ndarray) -> np.ndarray:
    """(U psi)_a = sum_b U_ab psi_b, per spin."""
    return np.einsum("...ab,...sb->...sa", u, psi)


def colour_mul_dag(u: np.ndarray, psi: np.ndarray) -> np.ndarray:
    """(U^dagger psi)_a = sum_b conj(U_ba) psi_b, per spin."""
    return np.einsum("...ba,...sb->...sa", u.conj(), psi)


def apply_gamma5(psi: np.ndarray) -> np.ndarray:
    return spin_mul(GAMMA5, psi)


def apply_dw(u: np.ndarray, psi: np.ndarray, mu: float, m_w: float) -> np.ndarray:
    """D_w(mu) psi, term by term as in Eq. WD_op."""
    kappa = kappa_of(m_w)
    out = psi.copy()
    for nu in range(4):
        f = hop_factor(nu, mu)
        u_nu = u[..., nu, :, :]
        g_plus = spin_mul(ID4 + GAMMA[nu], colour_mul(u_nu, shift(psi, nu, +1)))
        g_minus = spin_mul(ID4 - GAMMA[nu],
                           colour_mul_dag(shift(u_nu, nu, -1), shift(psi, nu, -1)))
        out -= kappa * (f * g_plus + g_minus / f)
    return out


def apply_dw_dagger(u: np.ndarray, psi: np.ndarray, mu: float, m_w: float) -> np.ndarray:
    """D_w(mu)^dagger psi from the explicit adjoint of each hopping term.

    (G_nu^+)^dagger psi (y) = (1 + gamma_nu) U_nu(y - nu)^dagger psi(y - nu)
    (G_nu^-)^dagger psi (y) = (1 - gamma_nu) U_nu(y) psi(y + nu)
    (gamma_nu is Hermitian, mu and kappa are real).
    """
    kappa = kappa_of(m_w)
    out = psi.copy()
    for nu in range(4):
        f = hop_factor(nu, mu)
        u_nu = u[..., nu, :, :]
        gp_dag = spin_mul(ID4 + GAMMA[nu],
                          colour_mul_dag(shift(u_nu, nu, -1), shift(psi, nu, -1)))
        gm_dag = spin_mul(ID4 - GAMMA[nu], colour_mul(u_nu, shift(psi, nu, +1)))
        out -= kappa * (f * gp_dag + gm_dag / f)
    return out


def apply_h(u, psi, mu, m_w):
    """H psi = gamma5 D_w(mu) psi (Sec. 1)."""
    return apply_gamma5(apply_dw(u, psi, mu, m_w))


def apply_h_dagger(u, psi, mu, m_w):
    """H^dagger psi = D_w(mu)^dagger gamma5 psi."""
    return apply_dw_dagger(u, apply_gamma5(psi), mu, m_w)


def apply_dh_dmu(u, psi, mu, m_w):
    """(dH/dmu) psi = -kappa gamma5 (e^{mu} G_4^+ - e^{-mu} G_4^-) psi (Eq. WD_op, d/dmu)."""
    kappa = kappa_of(m_w)
    nu = 3
    u_nu = u[..., nu, :, :]
    g_plus = spin_mul(ID4 + GAMMA[nu], colour_mul(u_nu, shift(psi, nu, +1)))
    g_minus = spin_mul(ID4 - GAMMA[nu],
                       colour_mul_dag(shift(u_nu, nu, -1), shift(psi, nu, -1)))
    return apply_gamma5(-kappa * (np.exp(mu) * g_plus - np.exp(-mu) * g_minus))


def apply_dh_dmu_dagger(u, psi, mu, m_w):
    """(dH/dmu)^dagger psi = (d D_w/dmu)^dagger gamma5 psi, from the explicit adjoint of
    the temporal hops: (G_4^+)^dag psi (y) = (1+gamma_4) U_4(y-t)^dag psi(y-t) and
    (G_4^-)^dag psi (y) = (1-gamma_4) U_4(y) psi(y+t)."""
    kappa = kappa_of(m_w)
    nu = 3
    u_nu = u[..., nu, :, :]
    phi = apply_gamma5(psi)
    gp_dag = spin_mul(ID4 + GAMMA[nu], colour_mul_dag(shift(u_nu, nu, -1), shift(phi, nu, -1)))
    gm_dag = spin_mul(ID4 - GAMMA[nu], colour_mul(u_nu, shift(phi, nu, +1)))
    return -kappa * (np.exp(mu) * gp_dag - np.exp(-mu) * gm_dag)


def apply_dh(u, e, psi, mu, m_w, m_dir):
    """Directional derivative d/dt H(U + t E, mu + t m) psi at t = 0 (Eq. WD_op is affine
    in the links, so the link part is the hopping part of D_w with E in place of U)."""
    out = m_dir * apply_dh_dmu(u, psi, mu, m_w) if m_dir else np.zeros_like(psi)
    if e is not None:
        out = out + apply_gamma5(apply_dw(e, psi, mu, m_w) - psi)
    return out


def apply_dh_dagger(u, e, psi, mu, m_w, m_dir):
    """Adjoint of ``apply_dh`` from the explicit adjoint of each term."""
    out = m_dir * apply_dh_dmu_dagger(u, psi, mu, m_w) if m_dir else np.zeros_like(psi)
    if e is not None:
        phi = apply_gamma5(psi)
        out = out + (apply_dw_dagger(e, phi, mu, m_w) - phi)
    return out


def link_gradient(a: np.ndarray, b: np.ndarray, u: np.ndarray, mu: float, m_w: float):
    """Contract a sum of rank-one terms g_H = sum_j a_j b_j^dagger into (dU, dmu).

    ``a`` and ``b`` are stacks (J, Nt, Nz, Ny, Nx, 4, 3).  The loss differential
    is dL = Re <g_H, dH>, with H depending on U through the hops of Eq. WD_G.
    The link gradient follows the complex (conjugate-Wirtinger) convention
    dL = Re sum conj(dU) * delta U over all 9 entries of every link.

    Forward hop, H_{(x,s,c),(x+nu,s',c')} = C+_{ss'} U_nu(x)_{cc'}:
        dU_nu(x)[c,c'] += sum_{s,s'} conj(C+_{ss'}) a_{x,s,c} conj(b_{x+nu,s',c'})
    Backward hop, H_{(x+nu,s,c),(x,s',c')} = C-_{ss'} (U_nu(x)^dagger)_{cc'}:
        M[c,c'] = sum_{s,s'} conj(C-_{ss'}) a_{x+nu,s,c} conj(b_{x,s',c'});  dU_nu(x) += M^dagger
    with C+ = -kappa f_nu gamma5 (1+gamma_nu), C- = -kappa f_nu^{-1} gamma5 (1-gamma_nu).
    dmu = Re sum_j <a_j, (dH/dmu) b_j>.
    """
    kappa = kappa_of(m_w)
    du = np.zeros_like(u)
    for nu in range(4):
        f = hop_factor(nu, mu)
        c_plus = -kappa * f * GAMMA5 @ (ID4 + GAMMA[nu])
        c_minus = -kappa / f * GAMMA5 @ (ID4 - GAMMA[nu])
        b_fwd = shift(b, nu, +1)
        a_fwd = shift(a, nu, +1)
        du[..., nu, :, :] += np.einsum("st,j...sc,j...td->...cd",
                                       c_plus.conj(), a, b_fwd.conj())
        m = np.einsum("st,j...sc,j...td->...cd", c_minus.conj(), a_fwd, b.conj())
        du[..., nu, :, :] += np.swapaxes(m, -1, -2).conj()
    dmu = float(np.real(np.vdot(a, apply_dh_dmu(u, b, mu, m_w))))
    return du, dmu
