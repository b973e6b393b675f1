"""The host eigenvalue routine of the run diagnostics (ov_tridiag_eigenvalues):
Ritz values of TSL tridiagonals against numpy's dense eigenvalue solver (LAPACK
zgeev), and the special cases it must reproduce.  Runs without a GPU."""
import numpy as np
import pytest
from scipy.optimize import linear_sum_assignment

from oracle import tsl
from paper_1604_08057_gb300 import binding, build, inputs


@pytest.fixture(scope="module", autouse=True)
def _lib():
    binding.load(build.build())


def _match(a, b):
    """Largest distance between the two spectra under the best pairing."""
    cost = np.abs(a[:, None] - b[None, :])
    r, c = linear_sum_assignment(cost)
    return cost[r, c].max()


def _random_tsl_tridiag(k, rng):
    alpha = rng.standard_normal(k) + 1j * rng.standard_normal(k)
    omega = rng.standard_normal(k) + 1j * rng.standard_normal(k)
    delta = np.sqrt(np.abs(omega))
    beta = omega / delta
    beta[0], delta[0] = 0, 0
    return alpha, beta, delta


@pytest.mark.parametrize("k", [1, 2, 3, 17, 200])
def test_random_tridiagonals_match_dense_eig(k):
    rng = np.random.default_rng(100 + k)
    a, b, d = _random_tsl_tridiag(k, rng)
    want = np.linalg.eigvals(tsl.tridiag(a, b, d))
    got = binding.tridiag_eigenvalues(a, b, d)
    assert _match(got, want) <= 1e-10 * max(1.0, np.abs(want).max())


@pytest.mark.parametrize("m_w,mu,k", [(-2.0, 0.3, 60), (-1.0, 0.3, 120), (-2.0, 0.0, 80)])
def test_tsl_ritz_values_match_dense_eig(m_w, mu, k):
    """T_k of the oracle's TSL on a 3^4 lattice: the Ritz values of the physics
    points, including mu = 0 where T_k is Hermitian and its spectrum real."""
    dims = (3, 3, 3, 3)
    rng = np.random.default_rng(5)
    u = inputs.su3_links(dims, 0.3, rng)
    b = inputs.gaussian_spinors(dims, 1, rng)[0]
    f = tsl.tsl_forward(u, b, mu, m_w, k)
    want = np.linalg.eigvals(f.t)
    got = binding.tridiag_eigenvalues(f.alpha, f.beta, f.delta)
    scale = np.abs(want).max()
    assert _match(got, want) <= 1e-9 * scale
    assert abs(np.abs(got.real).min() - np.abs(want.real).min()) <= 1e-9 * scale
    if mu == 0.0:
        assert np.abs(got.imag).max() <= 1e-10 * scale


def test_diagonal_and_split_matrices():
    """A diagonal matrix (every off-diagonal zero) returns its diagonal; a zero in
    the middle of the off-diagonal splits the spectrum into its two blocks."""
    a = np.array([1 + 2j, -3 + 0.5j, 0.25 - 1j, 4.0 + 0j])
    z = np.zeros(4)
    got = binding.tridiag_eigenvalues(a, z.astype(complex), z)
    assert _match(got, a) == 0.0
    rng = np.random.default_rng(9)
    a, b, d = _random_tsl_tridiag(10, rng)
    b[5], d[5] = 0, 0
    t = tsl.tridiag(a, b, d)
    want = np.concatenate([np.linalg.eigvals(t[:5, :5]), np.linalg.eigvals(t[5:, 5:])])
    assert _match(binding.tridiag_eigenvalues(a, b, d), want) <= 1e-12 * np.abs(want).max()


def test_rejects_non_finite_input():
    a, b, d = _random_tsl_tridiag(5, np.random.default_rng(1))
    a[2] = np.nan
    with pytest.raises(binding.OVError) as exc:
        binding.tridiag_eigenvalues(a, b, d)
    assert exc.value.status == -6


@pytest.mark.parametrize("k", [1, 2, 5, 40, 300])
def test_tridiagonal_eigenvectors_right_and_left(k):
    """ov_tridiag_eigenvector: T y = theta y and z^dag T = theta z^dag for every
    eigenvalue of random TSL tridiagonals, unit norm, against the residual bound
    of a backward-stable solve (and numpy's eigenvectors up to phase)."""
    rng = np.random.default_rng(500 + k)
    a, b, d = _random_tsl_tridiag(k, rng)
    t = tsl.tridiag(a, b, d)
    theta = binding.tridiag_eigenvalues(a, b, d)
    nt = np.linalg.norm(t, 2)
    for th in theta[: min(k, 25)]:
        y = binding.tridiag_eigenvector(a, b, d, th)
        z = binding.tridiag_eigenvector(a, b, d, th, left=True)
        assert abs(np.linalg.norm(y) - 1) <= 1e-12 and abs(np.linalg.norm(z) - 1) <= 1e-12
        assert np.linalg.norm(t @ y - th * y) <= 1e-9 * nt
        assert np.linalg.norm(z.conj() @ t - th * z.conj()) <= 1e-9 * nt


def test_tridiagonal_eigenvectors_match_dense_eig():
    rng = np.random.default_rng(7)
    a, b, d = _random_tsl_tridiag(12, rng)
    t = tsl.tridiag(a, b, d)
    w, v = np.linalg.eig(t)
    for i in range(12):
        y = binding.tridiag_eigenvector(a, b, d, w[i])
        vi = v[:, i] / np.linalg.norm(v[:, i])
        phase = np.vdot(vi, y)
        assert abs(abs(phase) - 1) <= 1e-9
        assert np.linalg.norm(y - phase * vi) <= 1e-9


def test_tridiagonal_eigenvector_rejects_bad_arguments():
    a, b, d = _random_tsl_tridiag(4, np.random.default_rng(1))
    with pytest.raises(binding.OVError):
        binding.tridiag_eigenvector(a, b, d, np.nan)


@pytest.mark.parametrize("m", [1, 2, 5, 40, 150])
def test_hessenberg_eigen_matches_dense_eig(m):
    """ov_hessenberg_eigen on random complex upper Hessenberg matrices: the spectrum
    of LAPACK's zgeev and A y = mu y for every returned pair."""
    rng = np.random.default_rng(900 + m)
    a = np.triu(rng.standard_normal((m, m)) + 1j * rng.standard_normal((m, m)), -1)
    eig, vec = binding.hessenberg_eigen(a)
    want = np.linalg.eigvals(a)
    assert _match(eig, want) <= 1e-10 * max(1.0, np.abs(want).max())
    na = np.linalg.norm(a, 2)
    for i in range(m):
        assert abs(np.linalg.norm(vec[:, i]) - 1) <= 1e-12
        assert np.linalg.norm(a @ vec[:, i] - eig[i] * vec[:, i]) <= 1e-9 * na


def test_hessenberg_eigen_special_cases():
    # diagonal (already deflated), a Jordan-like 2 x 2 block, and a rejected full matrix
    d = np.diag([3.0 + 1j, -2.0, 0.5j])
    eig = binding.hessenberg_eigen(d, vectors=False)
    assert _match(eig, np.diag(d)) <= 1e-14
    j = np.array([[1.0, 1.0], [1e-20, 1.0]], dtype=complex)
    eig = binding.hessenberg_eigen(j, vectors=False)
    assert np.allclose(eig, [1.0, 1.0], atol=1e-9)
    with pytest.raises(binding.OVError):
        binding.hessenberg_eigen(np.ones((4, 4)))
