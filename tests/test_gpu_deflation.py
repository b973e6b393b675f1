"""Deflation on the GPU (Sec. 3) through the C ABI, with eigen-triples and their
derivatives from the oracle's dense eigendecomposition of a 2^4 lattice's H
(n = 192): the standard deflation of sgn(H) b and the generalised deflation of
Theorem 1's block matrix against the oracle's deflation (oracle/deflation.py),
the accuracy gained at fixed k against the exact sign, the l = 0 case against
the plain TSL, and the rejection of an eigenvalue on the imaginary axis."""
import numpy as np
import pytest
import torch

from oracle import deflation, overlap, tsl
from paper_1604_08057_gb300 import binding, inputs

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


def T(a):
    return torch.tensor(a, device=DEV)


def lattice_case(seed=11):
    dims, mu, m_w = (2, 2, 2, 2), 0.3, -2.0
    rng = np.random.default_rng(seed)
    u = inputs.su3_links(dims, 0.3, rng)
    b = inputs.gaussian_spinors(dims, 2, rng)
    e = inputs.su3_links(dims, 0.3, rng) - u
    return u, b, e, mu, m_w


def test_deflated_sign_matches_the_oracle_and_gains_accuracy():
    u, b, e, mu, m_w = lattice_case()
    l, k = 32, 60
    d = deflation.lattice_eigendata(u, mu, m_w, l)
    x = binding.tsl_sign_deflated(T(u), mu, m_w, T(b), k, d["lam"], T(d["R"]), T(d["L"])).cpu().numpy()
    lam, r, l_ = deflation.eigentriples(d["h"])
    sgn = r @ np.diag(np.sign(lam.real)) @ l_.conj().T
    plain = binding.tsl_sign(T(u), mu, m_w, T(b), k).cpu().numpy()
    for s in range(2):
        want = deflation.deflated_sign_lattice(u, b[s], mu, m_w, k, d["lam"], d["R"], d["L"])
        assert rel(x[s], want) <= 1e-9, (s, rel(x[s], want))
        exact = sgn @ b[s].ravel()
        assert 10 * rel(x[s].ravel(), exact) <= rel(plain[s].ravel(), exact)


def test_generalised_deflation_matches_the_oracle():
    u, b, e, mu, m_w = lattice_case(12)
    l, k, m_dir = 8, 40, 0.2
    d = deflation.lattice_eigendata(u, mu, m_w, l, e, m_dir)
    dx, x = binding.tsl_sign_jvp_deflated(T(u), mu, m_w, T(b), k, d["lam"], T(d["R"]), T(d["L"]), T(d["dR"]),
                                          T(d["dL"]), e=T(e), m_dir=m_dir)
    dx, x = dx.cpu().numpy(), x.cpu().numpy()
    for s in range(2):
        dx_o, x_o = deflation.deflated_block_lattice(u, b[s], mu, m_w, k, e, m_dir, d["lam"], d["R"], d["L"],
                                                     d["dR"], d["dL"])
        assert rel(x[s], x_o) <= 1e-9, (s, rel(x[s], x_o))
        assert rel(dx[s], dx_o) <= 1e-8, (s, rel(dx[s], dx_o))


def test_no_deflation_is_the_plain_tsl():
    u, b, e, mu, m_w = lattice_case(13)
    empty = torch.zeros((0, 2, 2, 2, 2, 4, 3), dtype=torch.complex128, device=DEV)
    x = binding.tsl_sign_deflated(T(u), mu, m_w, T(b), 30, np.zeros(0, complex), empty, empty)
    assert torch.equal(x, binding.tsl_sign(T(u), mu, m_w, T(b), 30))
    dx, x2 = binding.tsl_sign_jvp_deflated(T(u), mu, m_w, T(b), 30, np.zeros(0, complex), empty, empty, empty,
                                           empty, e=T(e), m_dir=0.1)
    dx0, x0 = binding.tsl_sign_jvp(T(u), mu, m_w, T(b), 30, e=T(e), m_dir=0.1)
    assert torch.equal(dx, dx0) and torch.equal(x2, x0)


def test_eigenvalue_on_the_imaginary_axis_is_rejected():
    u, b, e, mu, m_w = lattice_case(14)
    d = deflation.lattice_eigendata(u, mu, m_w, 2)
    lam = d["lam"].copy()
    lam[1] = 1j * abs(lam[1])
    with pytest.raises(binding.OVError) as ei:
        binding.tsl_sign_deflated(T(u), mu, m_w, T(b), 20, lam, T(d["R"]), T(d["L"]))
    assert ei.value.status == -4   # OV_ERR_SIGN_ILLPOSED: sgn is not defined on Re z = 0


def test_ritz_triples_match_the_oracle_and_deflate():
    """Ritz triples of a k = 170 forward pass on 2^4 (m_w = -1, n = 192; the
    eigenvalues smallest in |lambda| converge last): the accepted eigenvalues and
    spectral projectors equal the oracle's Ritz triples of the same pass, the
    residuals are what they claim (H applied independently), and deflating them
    makes a k = 40 TSL more accurate against the exact sign."""
    dims, mu, m_w, k = (2, 2, 2, 2), 0.3, -1.0, 170
    rng = np.random.default_rng(41)
    u = inputs.su3_links(dims, 0.3, rng)
    b = inputs.gaussian_spinors(dims, 1, rng)[0]
    ut, bt = T(u), T(b)
    binding.tsl_sign(ut, mu, m_w, bt, k)
    th, R, L, res = binding.ritz_triples(ut, mu, m_w, k, 8, 1e-4)
    assert len(th) >= 4 and np.all(res <= 1e-4)
    th_o, R_o, L_o, res_o = deflation.ritz_triples(tsl.tsl_forward(u, b, mu, m_w, k), u, mu, m_w, 8, 1e-4)
    probe = rng.standard_normal(192) + 1j * rng.standard_normal(192)
    Rn, Ln = R.cpu().numpy(), L.cpu().numpy()
    for i in range(len(th)):
        j = int(np.argmin(np.abs(th_o - th[i])))
        assert abs(th_o[j] - th[i]) <= 1e-8
        p_gpu = Rn[i].ravel() * np.vdot(Ln[i].ravel(), probe)
        p_or = R_o[j].ravel() * np.vdot(L_o[j].ravel(), probe)
        assert rel(p_gpu, p_or) <= 1e-6
        hr = binding.apply_H(ut, mu, m_w, R[i]).cpu().numpy()
        assert abs(np.linalg.norm(hr - th[i] * Rn[i]) / np.linalg.norm(Rn[i]) - res[i]) <= 1e-3 * res[i] + 1e-14
    lam, r, l_ = deflation.eigentriples(overlap.dense_h(u, mu, m_w))
    exact = (r @ np.diag(np.sign(lam.real)) @ l_.conj().T) @ b.ravel()
    plain = binding.tsl_sign(ut, mu, m_w, bt, 40).cpu().numpy()
    defl = binding.tsl_sign_deflated(ut, mu, m_w, bt, 40, th, R, L).cpu().numpy()
    assert rel(defl.ravel(), exact) < rel(plain.ravel(), exact)


def test_ritz_triples_need_a_matching_forward_pass():
    dims, mu, m_w = (2, 2, 2, 2), 0.3, -1.0
    rng = np.random.default_rng(42)
    u = inputs.su3_links(dims, 0.3, rng)
    b = inputs.gaussian_spinors(dims, 1, rng)[0]
    binding.tsl_sign(T(u), mu, m_w, T(b), 30)
    with pytest.raises(binding.OVError):
        binding.ritz_triples(T(u), mu, m_w, 31, 4, 1e-6)      # k differs from the last pass


def _separated(lam_all, lam, count, gap=0.01):
    """Indices of eigenvalues in lam whose distance to every other eigenvalue of H
    exceeds gap (the shifted solves are conditioned by the gap)."""
    sel = []
    for i, x in enumerate(lam):
        d = np.abs(lam_all - x)
        d = d[d > 0]
        if d.min() > gap:
            sel.append(i)
        if len(sel) == count:
            break
    return sel


def test_eigen_derivatives_match_the_oracle():
    """dlambda_i, dR_i, dL_i by shifted GMRES on the GPU against the oracle's
    first-order perturbation formulas from the full eigendecomposition (2^4,
    m_w = -2, random link direction and mu direction), for eigenvalues separated
    from the rest by more than 0.01."""
    u, b, e, mu, m_w = lattice_case(12)
    m_dir = 0.2
    d = deflation.lattice_eigendata(u, mu, m_w, 16, e, m_dir)
    lam_all, _, _ = deflation.eigentriples(d["h"])
    sel = _separated(lam_all, d["lam"], 3)
    assert len(sel) >= 2
    dlam, dR, dL, res = binding.eigen_derivatives(T(u), mu, m_w, d["lam"][sel], T(d["R"][sel]), T(d["L"][sel]),
                                                  e=T(e), m_dir=m_dir)
    assert np.all(res <= 1e-10)
    dR, dL = dR.cpu().numpy(), dL.cpu().numpy()
    for c, i in enumerate(sel):
        assert abs(dlam[c] - d["dlam"][i]) <= 1e-10 * max(1.0, abs(d["dlam"][i]))
        assert rel(dR[c], d["dR"][i]) <= 1e-7, (i, rel(dR[c], d["dR"][i]))
        assert rel(dL[c], d["dL"][i]) <= 1e-7, (i, rel(dL[c], d["dL"][i]))


def test_generalised_deflation_with_gpu_eigen_derivatives():
    """The full GPU route: eigen-derivatives by shifted solves, then the generalised
    deflation, against the oracle's deflation with its own eigen-data."""
    u, b, e, mu, m_w = lattice_case(15)
    m_dir, k = 0.1, 40
    d = deflation.lattice_eigendata(u, mu, m_w, 16, e, m_dir)
    lam_all, _, _ = deflation.eigentriples(d["h"])
    sel = _separated(lam_all, d["lam"], 4)
    lam, Rs, Ls = d["lam"][sel], d["R"][sel], d["L"][sel]
    dlam, dR, dL, res = binding.eigen_derivatives(T(u), mu, m_w, lam, T(Rs), T(Ls), e=T(e), m_dir=m_dir)
    dx, x = binding.tsl_sign_jvp_deflated(T(u), mu, m_w, T(b), k, lam, T(Rs), T(Ls), dR, dL, e=T(e), m_dir=m_dir)
    dx, x = dx.cpu().numpy(), x.cpu().numpy()
    for s in range(2):
        dx_o, x_o = deflation.deflated_block_lattice(u, b[s], mu, m_w, k, e, m_dir, lam, Rs, Ls,
                                                     d["dR"][sel], d["dL"][sel])
        assert rel(x[s], x_o) <= 1e-9
        assert rel(dx[s], dx_o) <= 1e-7


def test_shift_invert_arnoldi_finds_the_smallest_eigen_triples():
    """ov_eigen_smallest on 2^4 at m_w = -2 (n = 192): the 8 eigenvalues smallest in
    |lambda| of the dense eigendecomposition, their spectral projectors, small
    residuals, and a deflated TSL with them equal to one with the exact triples."""
    u, b, e, mu, m_w = lattice_case(16)
    rng = np.random.default_rng(61)
    start = inputs.gaussian_spinors((2, 2, 2, 2), 1, rng)[0]
    lam, R, L, res = binding.eigen_smallest(T(u), mu, m_w, 8, 64, T(start))
    assert len(lam) == 8 and np.all(res <= 1e-8), res
    lam_all, r, l_ = deflation.eigentriples(overlap.dense_h(u, mu, m_w))
    assert np.allclose(np.sort(np.abs(lam)), np.abs(lam_all[:8]), rtol=1e-9)
    probe = rng.standard_normal(192) + 1j * rng.standard_normal(192)
    Rn, Ln = R.cpu().numpy(), L.cpu().numpy()
    for i in range(8):
        j = int(np.argmin(np.abs(lam_all - lam[i])))
        assert abs(lam_all[j] - lam[i]) <= 1e-9 * abs(lam_all[j])
        p_gpu = Rn[i].ravel() * np.vdot(Ln[i].ravel(), probe)
        p_ex = r[:, j] * np.vdot(l_[:, j], probe)
        assert rel(p_gpu, p_ex) <= 1e-6
    d = deflation.lattice_eigendata(u, mu, m_w, 8)
    x_gpu_triples = binding.tsl_sign_deflated(T(u), mu, m_w, T(b), 40, lam, R, L).cpu().numpy()
    x_exact_triples = binding.tsl_sign_deflated(T(u), mu, m_w, T(b), 40, d["lam"], T(d["R"]), T(d["L"])).cpu().numpy()
    assert rel(x_gpu_triples, x_exact_triples) <= 1e-7
