"""The seeded input generators shared by the oracle and the CUDA path: the
distributions and structure they promise, and the workload table against the
configurations the benchmark and the parity tests name (lattices, link spread,
mu, m_w, sources, k)."""
import numpy as np

from paper_1604_08057_gb300 import inputs


def test_su3_links_are_special_unitary_and_near_one_for_small_eps():
    dims = (3, 2, 2, 4)
    u = inputs.su3_links(dims, 0.3, np.random.default_rng(1))
    assert u.shape == (4, 2, 2, 3, 4, 3, 3)
    eye = np.eye(3)
    assert np.abs(u @ np.swapaxes(u, -1, -2).conj() - eye).max() < 1e-13
    assert np.abs(np.linalg.det(u) - 1.0).max() < 1e-13
    # U = expm(i eps A): the distance to 1 grows with eps and vanishes at eps = 0
    near = inputs.su3_links(dims, 0.01, np.random.default_rng(1))
    far = inputs.su3_links(dims, 0.3, np.random.default_rng(1))
    assert np.abs(near - eye).max() < 0.1 < np.abs(far - eye).max()
    assert np.abs(inputs.su3_links(dims, 0.0, np.random.default_rng(1)) - eye).max() < 1e-13
    # seeded: the same generator state gives the same links
    assert np.array_equal(u, inputs.su3_links(dims, 0.3, np.random.default_rng(1)))


def test_gaussian_spinors_and_z2_noise_statistics():
    dims = (4, 4, 4, 4)
    rng = np.random.default_rng(2)
    b = inputs.gaussian_spinors(dims, 3, rng)
    assert b.shape == (3, 4, 4, 4, 4, 4, 3)
    n = b.size
    assert abs(b.mean()) < 5.0 / np.sqrt(n)
    assert abs(np.mean(np.abs(b) ** 2) - 1.0) < 5.0 / np.sqrt(n)       # E|z|^2 = 1
    assert abs(np.mean(b.real ** 2) - 0.5) < 5.0 / np.sqrt(n)
    eta = inputs.z2_noise(dims, 2, rng)
    assert eta.dtype == np.complex128 and np.all(np.abs(eta) == 1.0) and np.all(eta.imag == 0.0)
    assert abs(eta.real.mean()) < 5.0 / np.sqrt(eta.size)


def test_tridiagonal_coefficients_have_the_tsl_layout():
    a, b, d = inputs.tridiagonal_coefficients(50, np.random.default_rng(3), shift=1.5)
    assert a.shape == b.shape == d.shape == (50,)
    assert b[0] == 0 and d[0] == 0
    assert np.allclose(np.abs(b[1:]), d[1:])                # the TSL's split |beta_j| = delta_j
    assert np.all(d[1:] > 0)
    assert np.all(np.abs(np.abs(a.real) - 1.5) < 6.0)      # +-shift plus a Gaussian


def test_workloads_match_the_stated_configurations():
    w = inputs.WORKLOADS
    assert (w["4x4^3"].dims, w["4x4^3"].eps, w["4x4^3"].mu, w["4x4^3"].m_w, w["4x4^3"].nsrc, w["4x4^3"].k) == \
        ((4, 4, 4, 4), 0.3, 0.3, -2.0, 1, 200)
    assert (w["8x8^3"].dims, w["8x8^3"].eps, w["8x8^3"].mu, w["8x8^3"].m_w, w["8x8^3"].nsrc, w["8x8^3"].k) == \
        ((8, 8, 8, 8), 0.25, 0.2, -2.0, 4, 400)
    assert (w["14x14^3"].dims, w["14x14^3"].eps, w["14x14^3"].mu, w["14x14^3"].m_w, w["14x14^3"].nsrc,
            w["14x14^3"].k) == ((14, 14, 14, 14), 0.2, 0.3, -2.0, 1, 800)
    assert (w["6x18^3"].dims, w["6x18^3"].eps, w["6x18^3"].mu, w["6x18^3"].m_w, w["6x18^3"].nsrc,
            w["6x18^3"].k) == ((18, 18, 18, 6), 0.2, 0.5, -2.0, 16, 600)
    assert w["14x14^3"].volume * 12 == 460992                 # n for 14^4
    assert w["4x4^3"].volume * 12 == 3072


def test_uneven_batch_mixes_lattices_mu_and_k():
    links, probs = inputs.uneven_batch()
    assert len(probs) == 32
    assert {p["dims"] for p in probs} == {(8, 8, 8, 8), (12, 12, 12, 6), (14, 14, 14, 14)}
    assert {p["mu"] for p in probs} == {0.1, 0.3, 0.5}
    ks = [p["k"] for p in probs]
    assert min(ks) >= 300 and max(ks) <= 1000 and len(set(ks)) > 16
    for p in probs:
        assert p["m_w"] == -2.0
        assert p["b"].shape == inputs.lattice_shape(p["dims"]) + (4, 3)
        assert links[p["dims"]].shape == inputs.lattice_shape(p["dims"]) + (4, 3, 3)
