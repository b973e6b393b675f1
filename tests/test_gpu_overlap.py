"""The overlap operator, its solver and the U(1) current estimator on the GPU
(Sec. 1, Eq. overlap; Sec. 4.3) against the oracle (oracle/overlap.py), through
the C ABI.

* D_ov b and D_ov^dagger b against the oracle's TSL form on the same k, at the
  well-conditioned m_w = -1 (bar 1e-11) and at the workload mass m_w = -2 on
  4x4^3 (10x the TSL map's rounding floor, 1e-9).
* GMRES on a 2^4 lattice with k = n = 192 (the TSL is exact to ~1e-10 there)
  against the dense solve of the exact D_ov; on 3^4 at k = 200 the true
  residual of the returned x, recomputed with an independent application.
* The current estimator for fixed Z2 noise vectors against the oracle's
  two-VJP estimator with chi from the dense solve, and its mu companion.
"""
import numpy as np
import pytest
import torch

from oracle import overlap, tsl, vjp
from paper_1604_08057_gb300 import binding, inputs

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


def T(a):
    return torch.tensor(a, device=DEV)


@pytest.mark.parametrize("dims,mu,m_w,k,tol", [((3, 5, 2, 4), 0.3, -1.0, 40, 1e-11),
                                                ((4, 4, 4, 4), 0.3, -2.0, 200, 1e-9)])
def test_overlap_apply_parity(dims, mu, m_w, k, tol):
    rng = np.random.default_rng(71)
    u = inputs.su3_links(dims, 0.3, rng)
    b = inputs.gaussian_spinors(dims, 2, rng)
    for dagger in (False, True):
        got = binding.overlap_apply(T(u), mu, m_w, T(b), k, dagger=dagger).cpu().numpy()
        for s in range(2):
            want = overlap.apply_dov(u, b[s], mu, m_w, k, dagger=dagger)
            assert rel(got[s], want) <= tol, (dagger, s, rel(got[s], want))


@pytest.fixture(scope="module")
def small():
    dims = (2, 2, 2, 2)
    rng = np.random.default_rng(62)
    u = inputs.su3_links(dims, 0.4, rng)
    eta = inputs.z2_noise(dims, 2, rng)
    d = overlap.dense_dov(u, 0.3, -1.0)
    return dims, u, eta, d


def test_solver_against_dense_solve(small):
    dims, u, eta, d = small
    mu, m_w, k = 0.3, -1.0, 192
    for dagger in (False, True):
        x, it, res = binding.overlap_solve(T(u), mu, m_w, T(eta), k, dagger=dagger, tol=1e-11, maxit=400)
        a = d.conj().T if dagger else d
        for s in range(2):
            want = np.linalg.solve(a, eta[s].ravel()).reshape(eta[s].shape)
            assert rel(x[s].cpu().numpy(), want) <= 1e-8, (dagger, s, it, res, rel(x[s].cpu().numpy(), want))
        assert res <= 1e-11 and it > 0


def test_solver_true_residual_at_partial_krylov_size():
    """3^4, k = 200 (the TSL converged to ~1e-10 at m_w = -1): the reported residual
    holds when D_ov x is applied again independently."""
    dims, mu, m_w, k = (3, 3, 3, 3), 0.3, -1.0, 200
    rng = np.random.default_rng(63)
    u = inputs.su3_links(dims, 0.3, rng)
    rhs = inputs.z2_noise(dims, 1, rng)[0]
    x, it, res = binding.overlap_solve(T(u), mu, m_w, T(rhs), k, tol=1e-9, maxit=400)
    ax = binding.overlap_apply(T(u), mu, m_w, x, k).cpu().numpy()
    assert rel(ax, rhs) <= 2e-9, (rel(ax, rhs), res, it)
    assert rel(overlap.apply_dov(u, x.cpu().numpy(), mu, m_w, k), rhs) <= 5e-9


def test_current_estimator_parity(small):
    dims, u, eta, d = small
    mu, m_w, k = 0.3, -1.0, 192
    j, tr = binding.u1_current(T(u), mu, m_w, T(eta), k, tol=1e-12, maxit=400)
    j = j.cpu().numpy()
    want = np.zeros_like(j)
    tr_want = 0.0
    for s in range(2):
        chi = np.linalg.solve(d.conj().T, eta[s].ravel()).reshape(eta[s].shape)
        want += overlap.current_estimate(u, eta[s], chi, mu, m_w, k) / 2
        xb = overlap.gamma5(chi)
        f = tsl.tsl_forward(u, eta[s], mu, m_w, k)
        _, d1, _ = vjp.tsl_vjp(u, eta[s], mu, m_w, k, xb, fwd=f)
        _, d2, _ = vjp.tsl_vjp(u, eta[s], mu, m_w, k, 1j * xb, fwd=f)
        tr_want += (d1 + 1j * d2) / 2
    assert rel(j, want) <= 1e-7, rel(j, want)
    assert abs(tr - tr_want) <= 1e-7 * abs(tr_want), (tr, tr_want)
