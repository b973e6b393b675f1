"""Pins for the oracle's nested Krylov approximation of the k x k sign (Sec. 4.1, one nesting level).

What fixes the nested result independently of the oracle's own code:
* the spectral mapping z -> (z + 1/z)/2 of S = (T + T^{-1})/2 and sgn(S) = sgn(T)
  (eigendecomposition of T);
* the first Arnoldi coefficient e_1^dag S e_1 = (T_11 + (T^{-1})_11)/2, with
  (T^{-1})_11 from the continued fraction of a tridiagonal matrix (a closed form);
* basis independence: the Ritz approximation Q sgn(Q^dag S Q) Q^dag e_1 is the same
  for any orthonormal basis of the Krylov space (here: QR of the Krylov matrix);
* exactness when the Krylov space is complete (m = k, or an invariant subspace);
* the nested TSL equal to sgn(H) b from the dense eigendecomposition at k = m = n.
* Theorem 1's block TSL with the nested stage equal to the Daleckii-Krein Frechet
  derivative and sgn(H) b at k = 2n (also at inner size 80 of 384).
"""
import numpy as np

from oracle import dirac, ksign, nested, tsl
from paper_1604_08057_gb300 import inputs
from tests.dense_util import dense_from_apply, sign_eig


def _tridiag(k, rng, shift=0.0):
    """A complex tridiagonal T with the TSL's split |beta_j| = delta_j."""
    alpha = rng.standard_normal(k) + 1j * rng.standard_normal(k)
    alpha += shift * np.sign(rng.standard_normal(k))
    omega = rng.standard_normal(k) + 1j * rng.standard_normal(k)
    delta = np.sqrt(np.abs(omega))
    beta = omega / delta
    beta[0] = delta[0] = 0.0
    return tsl.tridiag(alpha, beta, delta)


def test_inner_matrix_maps_spectrum_and_keeps_sign():
    rng = np.random.default_rng(41)
    t = _tridiag(30, rng, shift=1.5)
    s = nested.inner_matrix(t)
    lam = np.linalg.eigvals(t)
    want = np.sort_complex(0.5 * (lam + 1.0 / lam))
    assert np.allclose(np.sort_complex(np.linalg.eigvals(s)), want, atol=1e-9)
    assert np.allclose(sign_eig(s), sign_eig(t), atol=1e-9)


def test_first_coefficient_from_continued_fraction():
    rng = np.random.default_rng(42)
    k = 25
    t = _tridiag(k, rng, shift=2.0)
    # (T^{-1})_11 = 1 / (a_1 - b_2 d_2 / (a_2 - b_3 d_3 / (a_3 - ...)))
    frac = t[k - 1, k - 1]
    for j in range(k - 2, -1, -1):
        frac = t[j, j] - t[j, j + 1] * t[j + 1, j] / frac
    want = 0.5 * (t[0, 0] + 1.0 / frac)
    _, h, _ = nested.arnoldi(nested.inner_matrix(t), 4)
    assert abs(h[0, 0] - want) <= 1e-12 * abs(want)


def test_ritz_approximation_is_basis_independent():
    rng = np.random.default_rng(43)
    k, m = 40, 6
    t = _tridiag(k, rng, shift=1.5)
    s = nested.inner_matrix(t)
    e1 = np.zeros(k, dtype=np.complex128)
    e1[0] = 1.0
    krylov = np.stack([np.linalg.matrix_power(s, i) @ e1 for i in range(m)], axis=1)
    p, _ = np.linalg.qr(krylov)
    want = p @ sign_eig(p.conj().T @ s @ p) @ (p.conj().T @ e1)
    got = nested.nested_sign_e1(t, m)
    assert np.linalg.norm(got - want) <= 1e-9 * np.linalg.norm(want)
    # the Arnoldi relation and orthonormality of the inner basis
    q, h, meff = nested.arnoldi(s, m)
    assert meff == m
    assert np.abs(q.conj().T @ q - np.eye(m)).max() < 1e-13
    assert np.abs((s @ q - q @ h)[:, :-1]).max() < 1e-12


def test_complete_inner_space_gives_the_sign():
    rng = np.random.default_rng(44)
    k = 50
    t = _tridiag(k, rng, shift=1.5)
    want = sign_eig(t)[:, 0]
    for m in (k, k + 10):
        assert np.linalg.norm(nested.nested_sign_e1(t, m) - want) < 1e-9


def test_invariant_subspace_stops_early_and_is_exact():
    rng = np.random.default_rng(45)
    k = 20
    t = _tridiag(k, rng, shift=1.5)
    t[2, 3] = t[3, 2] = 0.0                   # T = blockdiag(T_1 (3 x 3), T_2)
    q, h, meff = nested.arnoldi(nested.inner_matrix(t), 10)
    assert meff == 3
    want = sign_eig(t)[:, 0]
    assert np.linalg.norm(nested.nested_sign_e1(t, 10) - want) < 1e-10


def test_nesting_beats_truncation_on_a_tsl_tridiagonal():
    """The property the nesting exists for: at inner size m, the Ritz approximation on S
    is far closer to sgn(T_k) e_1 than the outer TSL stopped at m steps (T_m)."""
    rng = np.random.default_rng(46)
    dims = (3, 3, 3, 3)
    u = inputs.su3_links(dims, 0.3, rng)
    b = inputs.gaussian_spinors(dims, 1, rng)[0]
    k, m = 150, 50
    res = tsl.tsl_forward(u, b, 0.3, -2.0, k, rebiorth=1)
    full = ksign.sign_newton(res.t)[:, 0]
    err_nested = np.linalg.norm(nested.nested_sign_e1(res.t, m) - full) / np.linalg.norm(full)
    trunc = np.zeros(k, dtype=np.complex128)
    trunc[:m] = ksign.sign_newton(res.t[:m, :m])[:, 0]
    err_trunc = np.linalg.norm(trunc - full) / np.linalg.norm(full)
    assert err_nested < 1e-6
    assert err_trunc > 1e3 * err_nested


def test_nested_tsl_reaches_the_exact_sign():
    dims = (2, 2, 2, 2)                        # n = 192
    rng = np.random.default_rng(47)
    u = inputs.su3_links(dims, 0.5, rng)
    b = inputs.gaussian_spinors(dims, 1, rng)[0]
    mu, m_w = 0.3, -1.0
    h = dense_from_apply(lambda p: dirac.apply_h(u, p, mu, m_w), b.shape)
    exact = (sign_eig(h) @ b.ravel()).reshape(b.shape)
    n = b.size
    x, y, res = nested.nested_tsl(u, b, mu, m_w, n, n, rebiorth=1)
    assert np.linalg.norm(x - exact) / np.linalg.norm(exact) < 1e-9
    # a short inner space already matches the outer result at this well-separated point
    x40, _, _ = nested.nested_tsl(u, b, mu, m_w, 120, 40, rebiorth=1)
    full = tsl.tsl_forward(u, b, mu, m_w, 120, rebiorth=1).x
    assert np.linalg.norm(x40 - full) / np.linalg.norm(full) < 1e-8


def test_nested_block_tsl_reaches_the_exact_derivative():
    """Theorem 1 with the nested k x k stage (the paper's derivative route): at k = 2n
    the upper half equals the Daleckii-Krein Frechet derivative L_sgn(H, dH) b and the
    lower half sgn(H) b, already at an inner size well below k."""
    from tests.dense_util import frechet_sign_daleckii_krein
    dims = (2, 2, 2, 2)
    rng = np.random.default_rng(62)
    u = inputs.su3_links(dims, 0.4, rng)
    b = inputs.gaussian_spinors(dims, 1, rng)[0]
    e = rng.standard_normal(u.shape) + 1j * rng.standard_normal(u.shape)
    mu, m_w, m_dir = 0.3, -1.0, 0.7
    hm = dense_from_apply(lambda p: dirac.apply_h(u, p, mu, m_w), b.shape)
    dhm = dense_from_apply(lambda p: dirac.apply_dh(u, e, p, mu, m_w, m_dir), b.shape)
    exact_d = frechet_sign_daleckii_krein(hm, dhm) @ b.ravel()
    exact_x = sign_eig(hm) @ b.ravel()
    k = 2 * b.size
    for m in (80, k):
        dx, x, _ = nested.nested_block_tsl(u, b, mu, m_w, k, m, e, m_dir)
        assert np.linalg.norm(dx.ravel() - exact_d) <= 1e-10 * np.linalg.norm(exact_d), m
        assert np.linalg.norm(x.ravel() - exact_x) <= 1e-10 * np.linalg.norm(exact_x), m
