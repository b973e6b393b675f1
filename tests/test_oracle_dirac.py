"""Pins for the oracle's Wilson-Dirac operator (App. A, Eqs. WD_op, WD_G, dWD_op).

Each test checks the oracle against a fact that is independent of its code:
Clifford algebra, the momentum-space closed form of the free operator, a
constant U(1) background (a shifted momentum), gauge covariance, the
definition of the adjoint, gamma5-hermiticity, and finite differences.
"""
import numpy as np
import pytest

from oracle import dirac
from paper_1604_08057_gb300 import inputs
from tests.dense_util import gauge_transform_links, gauge_transform_spinor, random_gauge


def _rand_spinor(dims, rng):
    return inputs.gaussian_spinors(dims, 1, rng)[0]


def test_gamma_algebra():
    g = dirac.GAMMA
    for mu in range(4):
        assert np.allclose(g[mu], g[mu].conj().T)
        for nu in range(4):
            anti = g[mu] @ g[nu] + g[nu] @ g[mu]
            assert np.allclose(anti, 2.0 * np.eye(4) * (mu == nu))
        assert np.allclose(dirac.GAMMA5 @ g[mu] + g[mu] @ dirac.GAMMA5, 0)
    # chiral basis: gamma5 = diag(1, 1, -1, -1)
    assert np.allclose(dirac.GAMMA5, np.diag([1, 1, -1, -1]))


def _momentum_matrix(p, mu, m_w, theta=(0, 0, 0, 0)):
    """Free Wilson-Dirac operator at lattice momentum p (per direction x,y,z,t)."""
    kappa = 1.0 / (2 * m_w + 8)
    m = np.eye(4, dtype=complex)
    for nu in range(4):
        f = np.exp(mu) if nu == 3 else 1.0
        ph = np.exp(1j * (p[nu] + theta[nu]))
        m = m - kappa * (f * (np.eye(4) + dirac.GAMMA[nu]) * ph
                         + (np.eye(4) - dirac.GAMMA[nu]) * np.conj(ph) / f)
    return m


@pytest.mark.parametrize("dims,mu,theta", [((4, 3, 2, 5), 0.3, (0, 0, 0, 0)),
                                           ((3, 4, 4, 2), -0.7, (0.4, -1.1, 0.25, 0.9))])
def test_free_field_momentum_space(dims, mu, theta):
    """U = e^{i theta_nu} 1: D_w is diagonal in momentum with p_nu -> p_nu + theta_nu."""
    rng = np.random.default_rng(3)
    m_w = -2.0
    shape = inputs.lattice_shape(dims)
    u = np.zeros(shape + (4, 3, 3), dtype=complex)
    for nu in range(4):
        u[..., nu, :, :] = np.exp(1j * theta[nu]) * np.eye(3)
    psi = _rand_spinor(dims, rng)
    out = dirac.apply_dw(u, psi, mu, m_w)
    psi_k = np.fft.fftn(psi, axes=(0, 1, 2, 3))
    out_k = np.fft.fftn(out, axes=(0, 1, 2, 3))
    nx, ny, nz, nt = dims
    for it in range(nt):
        for iz in range(nz):
            for iy in range(ny):
                for ix in range(nx):
                    p = (2 * np.pi * ix / nx, 2 * np.pi * iy / ny,
                         2 * np.pi * iz / nz, 2 * np.pi * it / nt)
                    m = _momentum_matrix(p, mu, m_w, theta)
                    want = m @ psi_k[it, iz, iy, ix]
                    assert np.allclose(out_k[it, iz, iy, ix], want, atol=1e-11)


def test_gauge_covariance():
    """D_w[U^Omega] (Omega psi) = Omega D_w[U] psi for a random SU(3) gauge transform."""
    dims = (3, 4, 2, 3)
    rng = np.random.default_rng(11)
    u = inputs.su3_links(dims, 0.5, rng)
    psi = _rand_spinor(dims, rng)
    om = random_gauge(inputs.lattice_shape(dims), rng)
    lhs = dirac.apply_dw(gauge_transform_links(u, om), gauge_transform_spinor(psi, om), 0.4, -2.0)
    rhs = gauge_transform_spinor(dirac.apply_dw(u, psi, 0.4, -2.0), om)
    assert np.allclose(lhs, rhs, atol=1e-12)


def test_adjoint_dot_test_and_gamma5_hermiticity():
    dims = (4, 3, 3, 2)
    rng = np.random.default_rng(12)
    u = inputs.su3_links(dims, 0.6, rng)
    a, b = _rand_spinor(dims, rng), _rand_spinor(dims, rng)
    mu, m_w = 0.35, -2.0
    lhs = np.vdot(a, dirac.apply_h(u, b, mu, m_w))
    rhs = np.vdot(dirac.apply_h_dagger(u, a, mu, m_w), b)
    assert abs(lhs - rhs) <= 1e-13 * abs(lhs)
    # H(mu)^dagger = gamma5 D_w(-mu)
    h_dag = dirac.apply_h_dagger(u, a, mu, m_w)
    assert np.allclose(h_dag, dirac.apply_gamma5(dirac.apply_dw(u, a, -mu, m_w)), atol=1e-13)
    # at mu = 0 H is Hermitian
    assert np.allclose(dirac.apply_h(u, a, 0.0, m_w), dirac.apply_h_dagger(u, a, 0.0, m_w),
                       atol=1e-13)


def test_dh_dmu_finite_difference():
    dims = (2, 3, 3, 4)
    rng = np.random.default_rng(13)
    u = inputs.su3_links(dims, 0.5, rng)
    psi = _rand_spinor(dims, rng)
    mu, m_w, h = 0.2, -2.0, 1e-5
    fd = (dirac.apply_h(u, psi, mu + h, m_w) - dirac.apply_h(u, psi, mu - h, m_w)) / (2 * h)
    assert np.allclose(dirac.apply_dh_dmu(u, psi, mu, m_w), fd, atol=1e-9)


def test_link_gradient_finite_difference():
    """d/dt Re <a, H(U + tE, mu + t m) b> = Re <dU, E> + dmu * m."""
    dims = (3, 2, 3, 3)
    rng = np.random.default_rng(14)
    u = inputs.su3_links(dims, 0.5, rng)
    a = np.stack([_rand_spinor(dims, rng) for _ in range(3)])
    b = np.stack([_rand_spinor(dims, rng) for _ in range(3)])
    e = rng.standard_normal(u.shape) + 1j * rng.standard_normal(u.shape)
    mu, m_w, h = 0.3, -2.0, 1e-6
    du, dmu = dirac.link_gradient(a, b, u, mu, m_w)

    def loss(uu, mm):
        return sum(np.real(np.vdot(a[j], dirac.apply_h(uu, b[j], mm, m_w))) for j in range(3))

    fd_u = (loss(u + h * e, mu) - loss(u - h * e, mu)) / (2 * h)
    assert abs(fd_u - np.real(np.vdot(du, e))) <= 1e-7 * abs(fd_u)
    fd_mu = (loss(u, mu + h) - loss(u, mu - h)) / (2 * h)
    assert abs(fd_mu - dmu) <= 1e-7 * max(1.0, abs(fd_mu))
    # a single entry, to catch a transposed colour index
    for (site, nu, c, d) in [((1, 0, 1, 2), 0, 0, 2), ((2, 1, 0, 0), 3, 2, 1), ((0, 1, 1, 1), 2, 1, 0)]:
        e1 = np.zeros_like(u)
        e1[site + (nu, c, d)] = 1.0
        fd_re = (loss(u + h * e1, mu) - loss(u - h * e1, mu)) / (2 * h)
        fd_im = (loss(u + 1j * h * e1, mu) - loss(u - 1j * h * e1, mu)) / (2 * h)
        got = du[site + (nu, c, d)]
        assert abs(got.real - fd_re) < 1e-7 and abs(got.imag - fd_im) < 1e-7
