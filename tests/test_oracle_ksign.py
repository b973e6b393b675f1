"""Pins for the oracle's small-matrix sign and its Frechet adjoint (Sec. 2, Theorems 1-2)."""
import numpy as np
import pytest

from oracle import ksign
from tests.dense_util import frechet_sign_daleckii_krein, sign_eig


def _rand_matrix(m, rng, shift=0.0):
    a = (rng.standard_normal((m, m)) + 1j * rng.standard_normal((m, m))) / np.sqrt(m)
    return a + shift * np.eye(m)


@pytest.mark.parametrize("m", [5, 40, 120])
def test_sign_matches_spectral_form(m):
    rng = np.random.default_rng(m)
    a = _rand_matrix(m, rng)
    f = ksign.sign_newton(a)
    assert np.allclose(f, sign_eig(a), atol=1e-9)
    assert np.allclose(f @ f, np.eye(m), atol=1e-10)          # sgn(A)^2 = 1
    assert np.allclose(f @ a, a @ f, atol=1e-10)              # commutes with A


def test_sign_hermitian_and_tridiagonal():
    rng = np.random.default_rng(7)
    m = 60
    h = _rand_matrix(m, rng)
    h = h + h.conj().T
    lam, q = np.linalg.eigh(h)
    want = q @ np.diag(np.sign(lam)) @ q.conj().T
    assert np.allclose(ksign.sign_newton(h), want, atol=1e-11)
    # a complex tridiagonal matrix, the shape of T_k
    t = np.diag(rng.standard_normal(m) + 1j * rng.standard_normal(m))
    t += np.diag(rng.standard_normal(m - 1) + 1j * rng.standard_normal(m - 1), 1)
    t += np.diag(np.abs(rng.standard_normal(m - 1)), -1)
    assert np.allclose(ksign.sign_newton(t), sign_eig(t), atol=1e-8)


def test_frechet_adjoint_vs_daleckii_krein_and_fd():
    rng = np.random.default_rng(21)
    m = 30
    a = _rand_matrix(m, rng)
    g = _rand_matrix(m, rng)
    e = _rand_matrix(m, rng)
    lstar = ksign.frechet_adjoint_sign(a, g)
    # adjoint of L(A, .) is L(A^dagger, .): compare with Daleckii-Krein on A^dagger
    assert np.allclose(lstar, frechet_sign_daleckii_krein(a.conj().T, g), atol=1e-9)
    # Re <G, L(A, E)> = Re <L*(A, G), E>, with L(A, E) from central differences
    h = 1e-6
    fd = (ksign.sign_newton(a + h * e) - ksign.sign_newton(a - h * e)) / (2 * h)
    lhs = np.real(np.vdot(g, fd))
    rhs = np.real(np.vdot(lstar, e))
    assert abs(lhs - rhs) <= 1e-6 * abs(lhs)


def test_theorem1_block_upper_right_is_derivative():
    """sgn([[A, E], [0, A]]) has sgn(A) on the diagonal and L(A, E) top right (Theorem 1)."""
    rng = np.random.default_rng(22)
    m = 25
    a, e = _rand_matrix(m, rng), _rand_matrix(m, rng)
    blk = np.block([[a, e], [np.zeros((m, m)), a]])
    s = ksign.sign_newton(blk)
    assert np.allclose(s[:m, :m], sign_eig(a), atol=1e-9)
    assert np.allclose(s[m:, m:], sign_eig(a), atol=1e-9)
    assert np.allclose(s[m:, :m], 0, atol=1e-12)
    assert np.allclose(s[:m, m:], frechet_sign_daleckii_krein(a, e), atol=1e-8)
    # the block matrix has the spectrum of A, each eigenvalue twice (Sec. 3)
    ev_b = np.sort_complex(np.linalg.eigvals(blk))
    ev_a = np.sort_complex(np.repeat(np.linalg.eigvals(a), 2))
    assert np.allclose(ev_b, ev_a, atol=1e-5)


def test_theorem2_block_eigendecomposition_is_wrong():
    """Theorem 2: the block matrix is defective, so the eigendecomposition route fails."""
    rng = np.random.default_rng(23)
    m = 12
    a, e = _rand_matrix(m, rng), _rand_matrix(m, rng)
    blk = np.block([[a, e], [np.zeros((m, m)), a]])
    via_eig = sign_eig(blk)[:m, m:]
    exact = frechet_sign_daleckii_krein(a, e)
    assert np.linalg.norm(via_eig - exact) > 1e-3 * np.linalg.norm(exact)


VARIANTS = [("det", "stagnation"), ("det", "predicted"), ("norm", "stagnation"), ("norm", "predicted")]


@pytest.mark.parametrize("m", [5, 40, 120])
@pytest.mark.parametrize("scaling_kind,stop", VARIANTS)
def test_sign_variants_match_spectral_form(m, scaling_kind, stop):
    """Every scaling and stop rule converges to the spectral sign (Sec. 2, Eq. spectral_form)."""
    rng = np.random.default_rng(100 + m)
    a = _rand_matrix(m, rng)
    f = ksign.sign_newton(a, scaling_kind=scaling_kind, stop=stop)
    assert np.allclose(f, sign_eig(a), atol=1e-9)
    assert np.allclose(f @ f, np.eye(m), atol=1e-10)
    h = a + a.conj().T
    lam, q = np.linalg.eigh(h)
    want = q @ np.diag(np.sign(lam)) @ q.conj().T
    assert np.allclose(ksign.sign_newton(h, scaling_kind=scaling_kind, stop=stop), want, atol=1e-10)


def test_sign_variants_on_a_tsl_tridiagonal():
    """On T_k of the 4x4^3 workload (k = 200) the variants agree with the determinant-scaled
    iteration to the sign's own rounding level, and norm scaling with the predicted stop
    needs fewer inversions."""
    from oracle import tsl
    from paper_1604_08057_gb300 import inputs
    wl = inputs.WORKLOADS["4x4^3"]
    u, b, _ = inputs.make_inputs(wl, nsrc=1)
    res = tsl.tsl_forward(u, b[0], wl.mu, wl.m_w, wl.k, rebiorth=20, passes=1)
    ref, it_ref = ksign.sign_newton(res.t, return_iters=True)
    floor = np.linalg.norm(ref @ ref - np.eye(wl.k)) / np.sqrt(wl.k)
    iters = {}
    for scaling_kind, stop in VARIANTS:
        f, it = ksign.sign_newton(res.t, return_iters=True, scaling_kind=scaling_kind, stop=stop)
        iters[(scaling_kind, stop)] = it
        assert np.linalg.norm(f[:, 0] - ref[:, 0]) <= 10 * floor * np.linalg.norm(ref[:, 0])
        assert np.linalg.norm(f @ f - np.eye(wl.k)) / np.sqrt(wl.k) <= 10 * floor
    assert iters[("det", "stagnation")] == it_ref
    assert iters[("det", "predicted")] <= it_ref - 1
    assert iters[("norm", "predicted")] <= it_ref - 2


def test_sign_rejects_unknown_rules():
    with pytest.raises(ValueError):
        ksign.sign_newton(np.eye(3), scaling_kind="spectral")
    with pytest.raises(ValueError):
        ksign.sign_newton(np.eye(3), stop="never")
