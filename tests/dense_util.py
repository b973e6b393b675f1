"""Dense restatements used only to pin the oracle on tiny lattices.

Nothing here is a step of the method: these helpers build explicit matrices
from the oracle's own operator (by applying it to unit vectors) and evaluate
exact matrix functions through library eigendecompositions.
"""
import numpy as np
import scipy.linalg as sla


def dense_from_apply(apply, shape):
    """Matrix of a linear map on arrays of ``shape`` (by columns, unit vectors)."""
    n = int(np.prod(shape))
    m = np.zeros((n, n), dtype=np.complex128)
    for i in range(n):
        e = np.zeros(n, dtype=np.complex128)
        e[i] = 1.0
        m[:, i] = apply(e.reshape(shape)).ravel()
    return m


def sign_eig(a):
    """sgn(A) from the spectral form X diag(sgn Re lambda) X^{-1} (Sec. 2, Eq. spectral_form)."""
    lam, x = sla.eig(a)
    return x @ np.diag(np.sign(lam.real)) @ np.linalg.inv(x)


def frechet_sign_daleckii_krein(a, e):
    """L_sgn(A, E) by the Daleckii-Krein formula for diagonalisable A.

    With A = X diag(lam) X^{-1}:  L = X [ (X^{-1} E X) o D ] X^{-1},
    D_ij = (f(lam_i) - f(lam_j)) / (lam_i - lam_j), and f'(lam) = 0 on the diagonal
    because sgn is locally constant.
    """
    lam, x = sla.eig(a)
    xi = np.linalg.inv(x)
    f = np.sign(lam.real)
    dl = lam[:, None] - lam[None, :]
    same = np.isclose(f[:, None], f[None, :])
    d = np.where(same, 0.0, (f[:, None] - f[None, :]) / np.where(same, 1.0, dl))
    return x @ ((xi @ e @ x) * d) @ xi


def random_gauge(dims_shape, rng):
    """Random SU(3) gauge transformation Omega(x), shape (Nt,Nz,Ny,Nx,3,3)."""
    z = rng.standard_normal(dims_shape + (3, 3)) + 1j * rng.standard_normal(dims_shape + (3, 3))
    q, r = np.linalg.qr(z)
    d = np.diagonal(r, axis1=-2, axis2=-1)
    q = q * (d / np.abs(d))[..., None, :]
    det = np.linalg.det(q)
    return q / (det ** (1.0 / 3.0))[..., None, None]


def gauge_transform_links(u, omega):
    """U_nu(x) -> Omega(x) U_nu(x) Omega(x+nu)^dagger."""
    out = np.empty_like(u)
    for nu in range(4):
        om_fwd = np.roll(omega, -1, axis=3 - nu)
        out[..., nu, :, :] = omega @ u[..., nu, :, :] @ np.swapaxes(om_fwd, -1, -2).conj()
    return out


def gauge_transform_spinor(psi, omega):
    """psi(x) -> Omega(x) psi(x) per spin."""
    return np.einsum("...ab,...sb->...sa", omega, psi)
