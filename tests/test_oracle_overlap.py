"""Pins for the oracle's overlap operator and U(1) current estimator (Sec. 1,
Eq. overlap; Sec. 4.3, Eqs. lat_vec_cur and divergence_def), on 2^4 lattices
where the exact dense operator is available.

* D_ov b and D_ov^dagger b from the TSL at k = n reproduce the dense
  1 + gamma5 sgn(H) (Newton sign, itself pinned against the spectral form).
* Jacobi's formula: Tr(D_ov^{-1} dD_ov/dTheta) = d log det D_ov / dTheta, the
  latter from central differences of slogdet -- this pins the current's
  definition and the way Theta enters the links.
* Gauge invariance: the divergence of the exact currents vanishes at every site
  (the link orientation and the backward hop's conjugate phase).
* The VJP form of the one-noise-vector estimator, <gamma5 chi, d(sgn(H) eta)/dTheta>
  with chi = D_ov^{-dagger} eta, equals eta^dagger D_ov^{-1} (dD_ov/dTheta) eta
  formed from dense matrices.
* Over Z2 noise the estimator's mean approaches the exact trace.
"""
import numpy as np
import pytest

from oracle import overlap
from paper_1604_08057_gb300 import inputs

DIMS = (2, 2, 2, 2)
N = 192


@pytest.fixture(scope="module")
def field():
    rng = np.random.default_rng(61)
    u = inputs.su3_links(DIMS, 0.4, rng)
    b = inputs.gaussian_spinors(DIMS, 1, rng)[0]
    return u, b, rng


@pytest.mark.parametrize("mu,m_w", [(0.3, -1.0), (0.3, -2.0)])
def test_dov_matches_dense_at_full_krylov_size(field, mu, m_w):
    u, b, _ = field
    d = overlap.dense_dov(u, mu, m_w)
    for dagger in (False, True):
        got = overlap.apply_dov(u, b, mu, m_w, N, dagger=dagger)
        want = ((d.conj().T if dagger else d) @ b.ravel()).reshape(b.shape)
        assert np.linalg.norm(got - want) <= 1e-8 * np.linalg.norm(want), (dagger, m_w)


@pytest.mark.parametrize("mu", [0.0, 0.3])
def test_current_is_the_derivative_of_log_det(field, mu):
    u, _, _ = field
    for site, nu in (((0, 0, 0, 0), 0), ((1, 0, 1, 0), 3), ((0, 1, 1, 1), 2)):
        j = overlap.exact_current(u, mu, -1.0, site, nu)
        want = overlap.dlogdet_dtheta(u, mu, -1.0, site, nu)
        assert abs(j - want) <= 1e-6 * max(1.0, abs(want)), (site, nu, j, want)


def test_divergence_of_exact_currents_vanishes(field):
    """At one site x: the four outgoing links (x, nu) and the four incoming ones
    (x - nu, nu); their currents enter the divergence with + and - signs."""
    u, _, _ = field
    mu, m_w = 0.3, -1.0
    x = np.array([1, 0, 1, 1])              # (t, z, y, x) index of the site
    j = np.zeros(inputs.lattice_shape(DIMS) + (4,), dtype=np.complex128)
    for nu in range(4):
        back = x.copy()
        back[3 - nu] = (back[3 - nu] - 1) % DIMS[nu]
        for site in (tuple(x), tuple(back)):
            j[site + (nu,)] = overlap.exact_current(u, mu, m_w, site, nu)
    div = overlap.divergence(j)[tuple(x)]
    assert abs(div) <= 1e-6 * np.abs(j).max(), (div, np.abs(j).max())
    assert np.abs(j).max() > 1e-2          # the currents themselves do not vanish


def test_vjp_estimator_matches_dense_estimator(field):
    u, _, rng = field
    mu, m_w = 0.3, -1.0
    eta = inputs.z2_noise(DIMS, 1, rng)[0]
    d = overlap.dense_dov(u, mu, m_w)
    chi = np.linalg.solve(d.conj().T, eta.ravel()).reshape(eta.shape)
    j = overlap.current_estimate(u, eta, chi, mu, m_w, N)
    for site, nu in (((0, 0, 0, 0), 0), ((1, 1, 0, 1), 1), ((0, 1, 1, 0), 3)):
        h = 1e-5
        dd = (overlap.dense_dov(overlap.with_theta(u, site, nu, h), mu, m_w)
              - overlap.dense_dov(overlap.with_theta(u, site, nu, -h), mu, m_w)) / (2 * h)
        want = np.vdot(eta.ravel(), np.linalg.solve(d, dd @ eta.ravel()))
        assert abs(j[site + (nu,)] - want) <= 1e-6 * max(1.0, abs(want)), (site, nu)


def test_z2_estimator_mean_approaches_the_trace(field):
    u, _, rng = field
    mu, m_w = 0.3, -1.0
    site, nu = (1, 0, 0, 1), 1
    d = overlap.dense_dov(u, mu, m_w)
    h = 1e-5
    dd = (overlap.dense_dov(overlap.with_theta(u, site, nu, h), mu, m_w)
          - overlap.dense_dov(overlap.with_theta(u, site, nu, -h), mu, m_w)) / (2 * h)
    m = np.linalg.solve(d, dd)
    exact = np.trace(m)
    etas = inputs.z2_noise(DIMS, 400, rng).reshape(400, -1)
    est = np.array([np.vdot(e, m @ e) for e in etas])
    err = abs(est.mean() - exact)
    sigma = est.std() / np.sqrt(len(est))
    assert err <= 4 * sigma + 1e-12, (err, sigma)
