"""Nested TSL (Sec. 4.1, one nesting level) on the GPU against the oracle, through the C ABI.

The k x k stage alone (ov_tridiag_sign_nested) is compared with ``oracle.nested``
on the same tridiagonal, so only rounding order separates the two: 1e-10
relative.  Whole calls (ov_tsl_sign, ov_tsl_sign_jvp with options.nested) are
compared with the oracle's nested TSL at the tolerances of the plain TSL parity
tests (10x the map's rounding floor: 1e-9 at the 4x4^3 workload point, where a
1e-16 perturbation of b moves x by 1e-10; 1e-10 at m_w = -1).
"""
import contextlib

import numpy as np
import pytest
import torch

from oracle import ksign, nested, tsl
from paper_1604_08057_gb300 import binding, inputs

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


def T(a):
    return torch.tensor(a, device=DEV)


@contextlib.contextmanager
def nested_option(m):
    binding.nested_sign(m)
    try:
        yield
    finally:
        binding.nested_sign(0)


def coefficients(t):
    """(alpha, beta, delta) of a tridiagonal in the layout of ov_tsl_coefficients."""
    k = t.shape[0]
    alpha = np.diag(t).copy()
    beta = np.zeros(k, dtype=np.complex128)
    delta = np.zeros(k)
    beta[1:] = np.diag(t, 1)
    delta[1:] = np.diag(t, -1).real
    return alpha, beta, delta


def random_tridiag(k, seed, diag_scale=1.0):
    """A complex tridiagonal with the TSL's balanced split |beta_j| = delta_j."""
    rng = np.random.default_rng(seed)
    alpha = diag_scale * (rng.standard_normal(k) + 1j * rng.standard_normal(k) + 1.5 * np.sign(rng.standard_normal(k)))
    omega = rng.standard_normal(k) + 1j * rng.standard_normal(k)
    delta = np.sqrt(np.abs(omega))
    beta = omega / delta
    beta[0] = delta[0] = 0.0
    return tsl.tridiag(alpha, beta, delta)


_WORKLOAD = {}


def workload_t():
    """T_k of the 4x4^3 workload (eps 0.3, mu 0.3, m_w -2, k 200) from the oracle."""
    if "t" not in _WORKLOAD:
        rng = np.random.default_rng(501)
        u = inputs.su3_links((4, 4, 4, 4), 0.3, rng)
        b = inputs.gaussian_spinors((4, 4, 4, 4), 1, rng)[0]
        _WORKLOAD["u"], _WORKLOAD["b"] = u, b
        _WORKLOAD["t"] = tsl.tsl_forward(u, b, 0.3, -2.0, 200, rebiorth=1).t
    return _WORKLOAD["t"]


@pytest.mark.parametrize("m", [0, 40, 60, 100, 200, 260])
def test_stage_on_workload_tridiagonal(m):
    t = workload_t()
    a, b, d = coefficients(t)
    y, iters = binding.tridiag_sign_nested(a, b, d, m, beta0=2.5)
    want = 2.5 * (ksign.sign_newton(t)[:, 0] if m == 0 else nested.nested_sign_e1(t, m))
    assert rel(y, want) <= 1e-10, rel(y, want)
    assert iters > 0


# (k, m, diagonal scale, seed): the small diagonals make the LU exchange rows at 2 of 2,
# 27 of 36 and 148 of 299 steps; each case's rounding floor (the nested result's change
# under a 1e-15 relative perturbation of T, in the oracle) is below 1e-13
@pytest.mark.parametrize("k,m,diag_scale,seed", [(2, 4, 1.0, 602), (2, 1, 1.0, 602), (3, 3, 0.2, 603),
                                                 (37, 12, 0.2, 637), (300, 70, 1.0, 900), (300, 70, 0.5, 900),
                                                 (129, 129, 1.0, 729)])
def test_stage_ragged_sizes_and_interchanges(k, m, diag_scale, seed):
    """Sizes off every tile (rows per block 8, columns per block 128), m >= k, m = 1,
    and row interchanges in the tridiagonal LU."""
    t = random_tridiag(k, seed, diag_scale)
    a, b, d = coefficients(t)
    y, _ = binding.tridiag_sign_nested(a, b, d, m)
    want = nested.nested_sign_e1(t, m)
    assert rel(y, want) <= 1e-10, rel(y, want)


def test_stage_invariant_subspace_closes_early():
    t = random_tridiag(40, 640)
    t[4, 5] = t[5, 4] = 0.0                    # blockdiag(T_1 (5 x 5), T_2): K(S, e_1) has dimension 5
    a, b, d = coefficients(t)
    y, _ = binding.tridiag_sign_nested(a, b, d, 20)
    want = nested.nested_sign_e1(t, 20)
    assert rel(y, want) <= 1e-10, rel(y, want)
    from tests.dense_util import sign_eig
    assert rel(y, sign_eig(t)[:, 0]) <= 1e-10


def test_stage_singular_tridiagonal_is_ill_posed():
    t = np.diag([0.0, 1.0]).astype(np.complex128)    # a zero first column: the LU finds no pivot
    a, b, d = coefficients(t)
    with pytest.raises(binding.OVError) as err:
        binding.tridiag_sign_nested(a, b, d, 2)
    assert err.value.status == -4              # OV_ERR_SIGN_ILLPOSED


def test_tsl_sign_nested_matches_oracle_at_workload_point():
    workload_t()
    u, b = _WORKLOAD["u"], _WORKLOAD["b"]
    k, m = 200, 60
    want, _, _ = nested.nested_tsl(u, b, 0.3, -2.0, k, m, rebiorth=1)
    with nested_option(m):
        x, info = binding.tsl_sign(T(u), 0.3, -2.0, T(b), k, return_info=True)
    assert rel(x.cpu().numpy(), want) <= 1e-9, rel(x.cpu().numpy(), want)
    # and it is the full-sign result to within the nested approximation (5e-14 at m = 60 in the oracle)
    full = binding.tsl_sign(T(u), 0.3, -2.0, T(b), k).cpu().numpy()
    assert rel(x.cpu().numpy(), full) <= 1e-9


def test_tsl_sign_nested_multi_source():
    rng = np.random.default_rng(650)
    dims = (3, 5, 2, 4)
    u = inputs.su3_links(dims, 0.3, rng)
    b = inputs.gaussian_spinors(dims, 3, rng)
    k, m = 90, 30
    with nested_option(m):
        x = binding.tsl_sign(T(u), 0.3, -1.0, T(b), k).cpu().numpy()
    for s in range(3):
        want, _, _ = nested.nested_tsl(u, b[s], 0.3, -1.0, k, m, rebiorth=1)
        assert rel(x[s], want) <= 1e-10, (s, rel(x[s], want))


def test_block_tsl_nested_matches_oracle():
    """Theorem 1's block TSL (the paper's derivative route) with the nested k x k sign."""
    rng = np.random.default_rng(660)
    dims = (3, 3, 3, 3)
    u = inputs.su3_links(dims, 0.3, rng)
    b = inputs.gaussian_spinors(dims, 1, rng)[0]
    e = rng.standard_normal(u.shape) + 1j * rng.standard_normal(u.shape)
    mu, m_w, k, m, m_dir = 0.3, -1.0, 100, 40, 0.5
    with nested_option(m):
        dx, x = binding.tsl_sign_jvp(T(u), mu, m_w, T(b), k, T(e), m_dir)
    _, _, res = tsl.block_tsl(u, b, mu, m_w, k, e, m_dir)
    y = res.beta0 * nested.nested_sign_e1(res.t, m)
    z = sum(y[j] * res.v[j] for j in range(k))
    assert rel(dx.cpu().numpy(), z[0]) <= 1e-9, rel(dx.cpu().numpy(), z[0])
    assert rel(x.cpu().numpy(), z[1]) <= 1e-9, rel(x.cpu().numpy(), z[1])


def test_reverse_mode_refuses_nested():
    rng = np.random.default_rng(670)
    dims = (2, 2, 2, 2)
    u = inputs.su3_links(dims, 0.3, rng)
    b = inputs.gaussian_spinors(dims, 1, rng)[0]
    xbar = inputs.gaussian_spinors(dims, 1, rng)[0]
    with nested_option(20):
        with pytest.raises(binding.OVError) as err:
            binding.tsl_sign_vjp(T(u), 0.3, -1.0, T(b), 40, T(xbar))
    assert err.value.status == -1              # OV_ERR_INVALID_ARG
    # the context computes normally afterwards
    du, dmu, x = binding.tsl_sign_vjp(T(u), 0.3, -1.0, T(b), 40, T(xbar))
    assert np.isfinite(dmu) and torch.isfinite(du).all()


def test_nested_at_the_benchmark_workload():
    """14x14^3, k = 800, P = 60, one Gram-Schmidt pass (the benchmark's launch
    configuration), inner size 100: the GPU stage against the oracle's nested sign on
    the call's own T_k (1e-10, identical input), and x from the nested stage against x
    from the full k x k sign (bench: 5e-12; required 1e-9, 10x the map's floor)."""
    wl = inputs.WORKLOADS["14x14^3"]
    u, b, _ = inputs.make_inputs(wl)
    ut, bt = T(u), T(b)
    k, m, period, passes = wl.k, 100, 60, 1
    full = binding.tsl_sign(ut, wl.mu, wl.m_w, bt, k, "fp64", period, passes)
    a, bb, d = binding.tsl_coefficients(k, 0, "fp64", period, passes)
    y, _ = binding.tridiag_sign_nested(a, bb, d, m)
    want = nested.nested_sign_e1(tsl.tridiag(a, bb, d), m)
    assert rel(y, want) <= 1e-10, rel(y, want)
    binding.nested_sign(m, "fp64", period, passes)
    try:
        x = binding.tsl_sign(ut, wl.mu, wl.m_w, bt, k, "fp64", period, passes)
    finally:
        binding.nested_sign(0, "fp64", period, passes)
    assert rel(x.cpu().numpy(), full.cpu().numpy()) <= 1e-9
