"""Pins for the oracle's two-sided Lanczos approximation of sgn(H) b."""
import numpy as np
import pytest

from oracle import dirac, tsl
from paper_1604_08057_gb300 import inputs
from tests.dense_util import (dense_from_apply, gauge_transform_links,
                              gauge_transform_spinor, random_gauge, sign_eig)


def _setup(dims, eps, seed):
    rng = np.random.default_rng(seed)
    u = inputs.su3_links(dims, eps, rng)
    b = inputs.gaussian_spinors(dims, 1, rng)[0]
    return u, b, rng


def test_biorthogonality_and_lanczos_relation():
    dims = (3, 3, 3, 3)
    u, b, _ = _setup(dims, 0.3, 31)
    mu, m_w, k = 0.3, -2.0, 60
    res = tsl.tsl_forward(u, b, mu, m_w, k, rebiorth=1)
    vm = np.stack([a.ravel() for a in res.v], 1)
    wm = np.stack([a.ravel() for a in res.w], 1)
    assert np.abs(wm.conj().T @ vm - np.eye(k)).max() < 1e-12
    hv = np.stack([dirac.apply_h(u, a, mu, m_w).ravel() for a in res.v], 1)
    resid = hv - vm @ res.t
    # only the last column may differ (by delta_{k+1} v_{k+1})
    assert np.abs(resid[:, :-1]).max() < 1e-12
    # and the left recurrence: H^dagger W = W T^dagger + ...
    hw = np.stack([dirac.apply_h_dagger(u, a, mu, m_w).ravel() for a in res.w], 1)
    assert np.abs((hw - wm @ res.t.conj().T)[:, :-1]).max() < 1e-12
    # y solves the projected problem: x = V y and y = beta0 sgn(T) e1
    assert np.allclose(res.x.ravel(), vm @ res.y)


def test_hermitian_case_mu_zero():
    """At mu = 0, H is Hermitian: w_j = v_j and the coefficients are real, beta = delta."""
    dims = (2, 3, 2, 3)
    u, b, _ = _setup(dims, 0.4, 32)
    res = tsl.tsl_forward(u, b, 0.0, -2.0, 40, rebiorth=1)
    for a, c in zip(res.v, res.w):
        assert np.allclose(a, c, atol=1e-12)
    assert np.abs(res.alpha.imag).max() < 1e-12
    assert np.allclose(res.beta[1:], res.delta[1:], atol=1e-12)


def test_converges_to_exact_sign_as_k_reaches_n():
    """With k = n the Krylov space is the whole space and TSL equals sgn(H) b exactly."""
    dims = (2, 2, 2, 2)                     # n = 192
    u, b, _ = _setup(dims, 0.5, 33)
    mu, m_w = 0.3, -1.0                     # spectrum well away from Re z = 0
    shape = b.shape
    h = dense_from_apply(lambda p: dirac.apply_h(u, p, mu, m_w), shape)
    exact = (sign_eig(h) @ b.ravel()).reshape(shape)
    n = b.size
    errs = {}
    for k in (40, 100, n):
        x = tsl.tsl_forward(u, b, mu, m_w, k, rebiorth=1).x
        errs[k] = np.linalg.norm(x - exact) / np.linalg.norm(exact)
    assert errs[n] < 1e-10
    assert errs[40] > errs[100] > errs[n]
    # the a-posteriori estimate (Eq. error_est) is small once converged
    assert tsl.eps_a(u, b, mu, m_w, n, rebiorth=1) < 1e-10


def test_gauge_covariance_of_tsl():
    """Coefficients are gauge invariant, x rotates with Omega."""
    dims = (3, 2, 2, 3)
    u, b, rng = _setup(dims, 0.4, 34)
    om = random_gauge(inputs.lattice_shape(dims), rng)
    mu, m_w, k = 0.25, -2.0, 30
    r0 = tsl.tsl_forward(u, b, mu, m_w, k)
    r1 = tsl.tsl_forward(gauge_transform_links(u, om), gauge_transform_spinor(b, om), mu, m_w, k)
    assert np.allclose(r0.alpha, r1.alpha, atol=1e-11)
    assert np.allclose(r0.beta, r1.beta, atol=1e-11)
    assert np.allclose(r0.delta, r1.delta, atol=1e-11)
    assert np.allclose(gauge_transform_spinor(r0.x, om), r1.x, atol=1e-10)


def test_rebiorth_schedules_agree_and_fp32_emulation_is_close():
    dims = (3, 3, 3, 3)
    u, b, _ = _setup(dims, 0.3, 35)
    mu, m_w, k = 0.3, -1.0, 50
    x_full = tsl.tsl_forward(u, b, mu, m_w, k, rebiorth=1).x
    x_pair = tsl.tsl_forward(u, b, mu, m_w, k, rebiorth=10).x
    x_cgs1 = tsl.tsl_forward(u, b, mu, m_w, k, rebiorth=1, passes=1).x
    nx = np.linalg.norm(x_full)
    assert np.linalg.norm(x_pair - x_full) / nx < 1e-9
    assert np.linalg.norm(x_cgs1 - x_full) / nx < 1e-10
    x32 = tsl.tsl_forward(u, b, mu, m_w, k, rebiorth=1, emulate_fp32=True).x
    err32 = np.linalg.norm(x32 - x_full) / nx
    assert 1e-9 < err32 < 1e-4


def test_rebiorth_schedule_definition():
    assert [j for j in range(1, 25) if tsl.rebiorth_at(j, 10)] == [1, 10, 11, 20, 21]
    assert all(tsl.rebiorth_at(j, 1) for j in range(1, 9))
    assert not any(tsl.rebiorth_at(j, 0) for j in range(1, 9))


def test_breakdown_is_reported():
    """b an exact eigenvector-free case: a source supported so that r = 0 at step 1."""
    dims = (2, 2, 2, 2)
    shape = inputs.lattice_shape(dims)
    u = np.zeros(shape + (4, 3, 3), dtype=complex)
    u[...] = np.eye(3)
    # the constant spinor with zero momentum is an eigenvector of the free H at mu = 0
    # only if gamma5 D_w maps it to a multiple of itself; use chirality to make it so:
    # at p = 0, D_w = 1 - 8 kappa (mu = 0), so H b = (1 - 8 kappa) gamma5 b, and a
    # chiral b (upper spins only) is an eigenvector.
    b = np.zeros(shape + (4, 3), dtype=complex)
    b[..., 0, 0] = 1.0
    with pytest.raises(tsl.Breakdown):
        tsl.tsl_forward(u, b, 0.0, -1.0, 5, rebiorth=0)
