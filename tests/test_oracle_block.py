"""Pins for the oracle's Theorem-1 block TSL (Sec. 2, Eq. func_derivative_1) and for
the directional derivative dH it uses."""
import numpy as np
import pytest

from oracle import dirac, tsl, vjp
from paper_1604_08057_gb300 import inputs
from tests.dense_util import dense_from_apply, frechet_sign_daleckii_krein, sign_eig


def _setup(dims, seed):
    rng = np.random.default_rng(seed)
    u = inputs.su3_links(dims, 0.4, rng)
    b = inputs.gaussian_spinors(dims, 1, rng)[0]
    e = rng.standard_normal(u.shape) + 1j * rng.standard_normal(u.shape)
    return u, b, e, rng


def test_dh_is_the_derivative_of_h_and_its_adjoint():
    u, b, e, rng = _setup((3, 2, 2, 3), 61)
    a = inputs.gaussian_spinors((3, 2, 2, 3), 1, rng)[0]
    mu, m_w, m = 0.3, -2.0, 0.7
    h = 1e-6
    fd = (dirac.apply_h(u + h * e, b, mu + h * m, m_w) - dirac.apply_h(u - h * e, b, mu - h * m, m_w)) / (2 * h)
    dh = dirac.apply_dh(u, e, b, mu, m_w, m)
    assert np.linalg.norm(fd - dh) <= 1e-9 * np.linalg.norm(dh)
    lhs = np.vdot(a, dh)
    rhs = np.vdot(dirac.apply_dh_dagger(u, e, a, mu, m_w, m), b)
    assert abs(lhs - rhs) <= 1e-13 * abs(lhs)
    # the mu part alone, and the links part alone
    assert np.allclose(dirac.apply_dh(u, None, b, mu, m_w, 1.0), dirac.apply_dh_dmu(u, b, mu, m_w))
    lhs = np.vdot(a, dirac.apply_dh(u, None, b, mu, m_w, 1.0))
    rhs = np.vdot(dirac.apply_dh_dmu_dagger(u, a, mu, m_w), b)
    assert abs(lhs - rhs) <= 1e-13 * abs(lhs)


@pytest.mark.parametrize("m_w", [-1.0, -2.0])
def test_block_tsl_is_exact_at_full_dimension(m_w):
    """With k = 2n the block Krylov space is the whole space: the upper half equals
    the Frechet derivative L_sgn(H, dH) b (Daleckii-Krein), the lower half sgn(H) b."""
    dims = (2, 2, 2, 2)
    u, b, e, _ = _setup(dims, 62)
    mu, m = 0.3, 0.7
    hm = dense_from_apply(lambda p: dirac.apply_h(u, p, mu, m_w), b.shape)
    dhm = dense_from_apply(lambda p: dirac.apply_dh(u, e, p, mu, m_w, m), b.shape)
    exact_d = frechet_sign_daleckii_krein(hm, dhm) @ b.ravel()
    exact_x = sign_eig(hm) @ b.ravel()
    dx, x, _ = tsl.block_tsl(u, b, mu, m_w, 2 * b.size, e, m)
    assert np.linalg.norm(dx.ravel() - exact_d) <= 1e-8 * np.linalg.norm(exact_d)
    assert np.linalg.norm(x.ravel() - exact_x) <= 1e-8 * np.linalg.norm(exact_x)


def test_block_tsl_converges_and_matches_the_vjp():
    dims = (2, 2, 2, 2)
    u, b, e, rng = _setup(dims, 63)
    xbar = inputs.gaussian_spinors(dims, 1, rng)[0]
    mu, m_w, m = 0.3, -1.0, 0.7
    hm = dense_from_apply(lambda p: dirac.apply_h(u, p, mu, m_w), b.shape)
    dhm = dense_from_apply(lambda p: dirac.apply_dh(u, e, p, mu, m_w, m), b.shape)
    exact_d = frechet_sign_daleckii_krein(hm, dhm) @ b.ravel()
    errs = []
    for k in (60, 250, 2 * b.size):
        dx, _, _ = tsl.block_tsl(u, b, mu, m_w, k, e, m)
        errs.append(np.linalg.norm(dx.ravel() - exact_d) / np.linalg.norm(exact_d))
    assert errs[0] > errs[1] > errs[2] and errs[2] < 1e-8
    # forward mode (Theorem 1) and reverse mode agree once both have converged
    dx, _, _ = tsl.block_tsl(u, b, mu, m_w, 2 * b.size, e, m)
    du, dmu, _ = vjp.tsl_vjp(u, b, mu, m_w, 190, xbar)
    jvp = np.real(np.vdot(xbar, dx))
    assert abs(jvp - (np.real(np.vdot(du, e)) + dmu * m)) <= 1e-6 * abs(jvp)


def test_block_tsl_left_start_reading():
    """w_1 = v_1 = (0, b) keeps the left space in the lower half (T_k = plain TSL's);
    the reading w_1 = (b, b)/||b|| is needed for a derivative."""
    dims = (2, 2, 2, 2)
    u, b, e, _ = _setup(dims, 64)
    mu, m_w, k = 0.3, -1.0, 40
    _, _, res = tsl.block_tsl(u, b, mu, m_w, k, e, 0.5)
    plain = tsl.tsl_forward(u, b, mu, m_w, k)
    assert np.abs(res.alpha - plain.alpha).max() > 1e-3


@pytest.mark.parametrize("m_w", [-1.0, -2.0])
def test_block_tsl_from_a_general_start_is_exact_at_full_dimension(m_w):
    """sgn(B) (t, l) = (sgn(H) t + L_sgn(H, dH) l, sgn(H) l) (Theorem 1) at k = 2n."""
    dims = (2, 2, 2, 2)
    u, b, e, rng = _setup(dims, 65)
    t = inputs.gaussian_spinors(dims, 1, rng)[0]
    mu, m = 0.3, 0.7
    hm = dense_from_apply(lambda p: dirac.apply_h(u, p, mu, m_w), b.shape)
    dhm = dense_from_apply(lambda p: dirac.apply_dh(u, e, p, mu, m_w, m), b.shape)
    s = sign_eig(hm)
    want_top = s @ t.ravel() + frechet_sign_daleckii_krein(hm, dhm) @ b.ravel()
    want_bot = s @ b.ravel()
    zt, zb, _ = tsl.block_tsl_start(u, t, b, mu, m_w, 2 * b.size, e, m)
    assert np.linalg.norm(zt.ravel() - want_top) <= 1e-8 * np.linalg.norm(want_top)
    assert np.linalg.norm(zb.ravel() - want_bot) <= 1e-8 * np.linalg.norm(want_bot)


def test_eps_b_vanishes_at_full_dimension_and_decreases_with_k():
    dims = (2, 2, 2, 2)
    u, b, e, _ = _setup(dims, 66)
    mu, m_w, m = 0.3, -1.0, 0.7
    eps = [tsl.eps_b(u, b, mu, m_w, k, e, m) for k in (40, 120, 2 * b.size)]
    assert eps[0] > eps[1] > eps[2] and eps[2] < 1e-9, eps


def test_eps_b_reduces_to_eps_a_without_a_direction():
    """With dH = 0 the block matrix is diag(H, H): started from (0, b) the right
    space stays in the lower half and T_k is the plain TSL's, so the block estimate
    of Eq. bA_error_est equals eps_A of Eq. error_est."""
    dims = (2, 2, 2, 2)
    u, b, _, _ = _setup(dims, 67)
    mu, m_w, k = 0.3, -1.0, 50
    ea = tsl.eps_a(u, b, mu, m_w, k)
    eb = tsl.eps_b(u, b, mu, m_w, k, None, 0.0)
    assert ea > 1e-6 and abs(eb - ea) <= 1e-9 * ea, (ea, eb)
