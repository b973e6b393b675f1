"""Pins of the deflation oracle (Sec. 3, App. B) against the mathematics: the
eigen-triples' defining equations, eigenvalue and eigenvector derivatives
against central finite differences, the deflated sign and the generalised
deflation of Theorem 1's block matrix against the exact sign and the exact
Frechet derivative (Daleckii-Krein in the eigenbasis) when the Krylov space
exhausts the deflated complement, and deflation's gain in accuracy at fixed k
on a lattice operator."""
import numpy as np

from oracle import deflation, overlap, tsl
from paper_1604_08057_gb300 import inputs


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


def diag_matrix(n, seed):
    """A = X diag(lam) X^{-1} with eigenvalues |Re lam| in [0.4, 2] of both signs."""
    rng = np.random.default_rng(seed)
    re = rng.uniform(0.4, 2.0, n) * rng.choice([-1.0, 1.0], n)
    lam = re + 1j * rng.uniform(-1.0, 1.0, n)
    x = np.eye(n) + 0.3 * (rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))) / np.sqrt(n)
    return x @ np.diag(lam) @ np.linalg.inv(x), lam, x


def exact_sign_and_derivative(lam, x, da):
    xi = np.linalg.inv(x)
    s = np.sign(lam.real)
    sgn = x @ np.diag(s) @ xi
    m = xi @ da @ x
    gam = np.zeros_like(m)
    for i in range(len(lam)):
        for j in range(len(lam)):
            if s[i] != s[j]:
                gam[i, j] = (s[i] - s[j]) / (lam[i] - lam[j])
    return sgn, x @ (gam * m) @ xi


def test_eigentriples_are_biorthonormal_eigenvectors():
    rng = np.random.default_rng(3)
    a = rng.standard_normal((24, 24)) + 1j * rng.standard_normal((24, 24))
    lam, r, l_ = deflation.eigentriples(a)
    assert np.all(np.diff(np.abs(lam)) >= 0)
    assert np.linalg.norm(a @ r - r * lam) <= 1e-12 * np.linalg.norm(a) * 24
    assert np.linalg.norm(l_.conj().T @ a - lam[:, None] * l_.conj().T) <= 1e-10 * np.linalg.norm(a) * 24
    assert np.abs(l_.conj().T @ r - np.eye(24)).max() <= 1e-10


def test_eigen_derivatives_match_central_differences():
    rng = np.random.default_rng(4)
    n = 20
    a = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
    da = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
    lam, r, l_ = deflation.eigentriples(a)
    idx = [0, 3, 7]
    dlam, dr, dl = deflation.eigen_derivatives(lam, r, l_, da, idx)
    t = 1e-6
    for c, i in enumerate(idx):
        fd = {}
        for sgn in (+1, -1):
            lt, rt, ltl = deflation.eigentriples(a + sgn * t * da)
            j = int(np.argmin(np.abs(lt - lam[i])))
            ri = rt[:, j] / np.vdot(l_[:, i], rt[:, j])          # gauge <L_i(0)|R_i(t)> = 1
            li = ltl[:, j] / np.conj(np.vdot(ltl[:, j], ri))       # <L_i(t)|R_i(t)> = 1
            fd[sgn] = (lt[j], ri, li)
        assert abs((fd[1][0] - fd[-1][0]) / (2 * t) - dlam[c]) <= 1e-6 * max(1.0, abs(dlam[c]))
        assert rel((fd[1][1] - fd[-1][1]) / (2 * t), dr[:, c]) <= 1e-5
        assert rel((fd[1][2] - fd[-1][2]) / (2 * t), dl[:, c]) <= 1e-5
        assert abs(np.vdot(l_[:, i], dr[:, c])) <= 1e-10 * np.linalg.norm(dr[:, c])
        assert abs(np.vdot(dl[:, c], r[:, i])) <= 1e-10 * np.linalg.norm(dl[:, c])


def test_deflated_sign_exact_when_krylov_space_exhausts_the_complement():
    n, l = 40, 6
    a, lam, x = diag_matrix(n, 5)
    b = np.random.default_rng(6).standard_normal(n) + 0j
    lam_s, r, l_ = deflation.eigentriples(a)
    sgn, _ = exact_sign_and_derivative(lam, x, np.zeros((n, n)))
    got = deflation.deflated_sign_dense(a, b, n - l, lam_s[:l], r[:, :l], l_[:, :l])
    assert rel(got, sgn @ b) <= 1e-9


def test_generalised_deflation_exact_when_krylov_space_exhausts_the_complement():
    n, l = 24, 4
    a, lam, x = diag_matrix(n, 7)
    rng = np.random.default_rng(8)
    da = 0.5 * (rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n)))
    b = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    lam_s, r, l_ = deflation.eigentriples(a)
    idx = list(range(l))
    dlam, dr, dl = deflation.eigen_derivatives(lam_s, r, l_, da, idx)
    sgn, dsgn = exact_sign_and_derivative(lam, x, da)
    dx, xx = deflation.deflated_block_dense(a, da, np.zeros(n, complex), b, 2 * (n - l), lam_s[:l], r[:, :l],
                                            l_[:, :l], dr, dl)
    assert rel(xx, sgn @ b) <= 1e-8
    assert rel(dx, dsgn @ b) <= 1e-7


def test_no_deflation_is_the_plain_tsl():
    a, _, _ = diag_matrix(30, 9)
    b = np.random.default_rng(10).standard_normal(30) + 0j
    lam_s, r, l_ = deflation.eigentriples(a)
    got = deflation.deflated_sign_dense(a, b, 12, lam_s[:0], r[:, :0], l_[:, :0])
    want = tsl.tsl_forward_op(lambda v: a @ v, lambda v: a.conj().T @ v, b, 12).x
    assert np.array_equal(got, want)


def lattice_case(seed=11):
    dims, mu, m_w = (2, 2, 2, 2), 0.3, -2.0
    rng = np.random.default_rng(seed)
    u = inputs.su3_links(dims, 0.3, rng)
    b = inputs.gaussian_spinors(dims, 1, rng)[0]
    e = inputs.su3_links(dims, 0.3, rng) - u
    return u, b, e, mu, m_w


def test_deflation_gains_accuracy_at_fixed_k_on_the_lattice():
    """H = gamma5 D_w at m_w = -2 on 2^4 (n = 192, an eigenvalue 2.2e-3 from the
    imaginary axis): deflating the 32 eigenvalues smallest in |lambda| makes the
    k = 60 TSL at least 10x more accurate (measured: 1.0e-2 against 0.87)."""
    u, b, e, mu, m_w = lattice_case()
    d = deflation.lattice_eigendata(u, mu, m_w, 32)
    lam, r, l_ = deflation.eigentriples(d["h"])
    exact = (r @ np.diag(np.sign(lam.real)) @ l_.conj().T) @ b.ravel()
    plain = tsl.tsl_forward(u, b, mu, m_w, 60).x
    defl = deflation.deflated_sign_lattice(u, b, mu, m_w, 60, d["lam"], d["R"], d["L"])
    e_plain, e_defl = rel(plain.ravel(), exact), rel(defl.ravel(), exact)
    assert e_defl * 10 <= e_plain, (e_defl, e_plain)


def test_lattice_forms_agree_with_the_dense_forms():
    u, b, e, mu, m_w = lattice_case(12)
    d = deflation.lattice_eigendata(u, mu, m_w, 8, e, 0.2)
    nl = 8
    r, l_ = d["R"].reshape(nl, -1).T, d["L"].reshape(nl, -1).T
    dr, dl = d["dR"].reshape(nl, -1).T, d["dL"].reshape(nl, -1).T
    x_lat = deflation.deflated_sign_lattice(u, b, mu, m_w, 24, d["lam"], d["R"], d["L"])
    x_den = deflation.deflated_sign_dense(d["h"], b.ravel(), 24, d["lam"], r, l_)
    assert rel(x_lat.ravel(), x_den) <= 1e-10
    dx_lat, xb_lat = deflation.deflated_block_lattice(u, b, mu, m_w, 24, e, 0.2, d["lam"], d["R"], d["L"],
                                                      d["dR"], d["dL"])
    dx_den, xb_den = deflation.deflated_block_dense(d["h"], d["dh"], np.zeros(b.size, complex), b.ravel(), 24,
                                                    d["lam"], r, l_, dr, dl)
    assert rel(xb_lat.ravel(), xb_den) <= 1e-10
    assert rel(dx_lat.ravel(), dx_den) <= 1e-9


def test_ritz_triples_of_a_full_krylov_space_are_the_eigen_triples():
    """With k = n (the 2^4 lattice, n = 192, m_w = -1 where the TSL reaches k = n),
    the Ritz triples of the TSL are H's eigen-triples: the same eigenvalues, and
    the same spectral projectors R_i <L_i| as the dense eigendecomposition."""
    dims, mu, m_w = (2, 2, 2, 2), 0.3, -1.0
    rng = np.random.default_rng(21)
    u = inputs.su3_links(dims, 0.3, rng)
    b = inputs.gaussian_spinors(dims, 1, rng)[0]
    fwd = tsl.tsl_forward(u, b, mu, m_w, 192)
    th, R, L, res = deflation.ritz_triples(fwd, u, mu, m_w, 10, 1e-8)
    assert len(th) == 10 and np.all(res <= 1e-8)
    lam, r, l_ = deflation.eigentriples(overlap.dense_h(u, mu, m_w))
    probe = rng.standard_normal(192) + 1j * rng.standard_normal(192)
    for i in range(10):
        j = int(np.argmin(np.abs(lam - th[i])))
        assert abs(lam[j] - th[i]) <= 1e-9 * abs(lam).max()
        p_ritz = R[i].ravel() * np.vdot(L[i].ravel(), probe)
        p_eig = r[:, j] * np.vdot(l_[:, j], probe)
        assert rel(p_ritz, p_eig) <= 1e-7
