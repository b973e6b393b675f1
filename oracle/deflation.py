"""Deflation of the sign function and of its derivative (test infrastructure).

Sec. 3: deflating the eigenvalues of H smallest in absolute value speeds up the
TSL approximation.  For the sign itself (standard deflation, H diagonalisable):

    sgn(H) b = sgn(H) Pbar b + sum_i sgn(lambda_i) R_i <L_i|b>,
    Pbar = 1 - sum_{i<=l} |R_i><L_i|,

with right and left eigenvectors R_i, L_i (H R_i = lambda_i R_i,
<L_i| H = lambda_i <L_i|, <L_i|R_j> = delta_ij) and sgn(lambda) = sgn(Re lambda);
the first term is the TSL approximation of sgn(H) applied to Pbar b.

For the block matrix B = [[H, dH], [0, H]] of Theorem 1, which is not
diagonalisable (the theorem of Sec. 3: its Jordan blocks have size two), the
generalised deflation of Sec. 3 (Eqs.
xinv_final, x_final, projector_1, defl_res_1, final_res) uses the columns x_i
of the Jordan transformation X and the rows xbar_i of X^{-1}:

    x_{2i-1} = (R_i, 0),   x_{2i} = (dR_i, R_i) / dlambda_i,
    xbar_{2i-1} = (<L_i|, <dL_i|),   xbar_{2i} = dlambda_i (0, <L_i|),

so that for psi = (top, bottom), with the 1/dlambda_i factors cancelling,

    P_{2l} psi = sum_i [ (R_i, 0) (<L_i|top> + <dL_i|bottom>) + (dR_i, R_i) <L_i|bottom> ],
    sgn(B) psi = sgn(B) (psi - P_{2l} psi)                       (TSL on the block matrix)
               + sum_i sgn(lambda_i) [ same terms as P_{2l} psi ]  (exact part),

the mixing term d sgn(lambda_i) of Eq. final_res being zero for the sign
(no eigenvalue crosses Re z = 0 along the direction).  The eigenvector
derivatives dR_i, dL_i are those of App. B, normalised by <L_i|dR_i> = 0 and
<dL_i|R_i> = 0; here they come from the full eigendecomposition (first-order
perturbation theory), the plain definition the paper's shifted inversions
compute:  with M = L^dag dH R,

    dlambda_i = M_ii,   dR_i = sum_{j != i} R_j M_ji / (lambda_i - lambda_j),
    d<L_i| = sum_{j != i} M_ij / (lambda_i - lambda_j) <L_j|.

Only tests/ and bench.py's reference legs use this module.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla

from . import overlap, tsl


def eigentriples(a: np.ndarray):
    """All eigenvalues and biorthonormal right / left eigenvectors of a dense matrix:
    (lam, R, L) with a R = R diag(lam), L^dag a = diag(lam) L^dag, L^dag R = 1,
    every R_i of unit norm.  Sorted by |lambda| ascending."""
    lam, vl, vr = sla.eig(np.asarray(a, dtype=np.complex128), left=True, right=True)
    order = np.argsort(np.abs(lam), kind="stable")
    lam, vl, vr = lam[order], vl[:, order], vr[:, order]
    r = vr / np.linalg.norm(vr, axis=0, keepdims=True)
    s = np.einsum("ij,ij->j", vl.conj(), r)          # <vl_i|R_i>
    l_ = vl / s.conj()[None, :]
    return lam, r, l_


def eigen_derivatives(lam, r, l_, da, idx):
    """dlambda_i, dR_i, dL_i (kets) for the eigenvalues idx, along the perturbation
    da, from the full biorthonormal eigendecomposition (App. B)."""
    m = l_.conj().T @ np.asarray(da, dtype=np.complex128) @ r
    dlam = np.array([m[i, i] for i in idx])
    dr = np.zeros((r.shape[0], len(idx)), dtype=np.complex128)
    dl = np.zeros_like(dr)
    for c, i in enumerate(idx):
        diff = lam[i] - lam
        mask = np.arange(len(lam)) != i
        dr[:, c] = r[:, mask] @ (m[mask, i] / diff[mask])
        dl_bra = (m[i, mask] / diff[mask]) @ l_[:, mask].conj().T      # d<L_i| as a row
        dl[:, c] = dl_bra.conj()
    return dlam, dr, dl


def projector_terms(top, bottom, r, l_, dr=None, dl=None):
    """The coefficient vectors of P_{2l} psi for psi = (top, bottom) (Eq. projector_1 with
    the columns / rows of Eqs. x_final, xinv_final): a_i = <L_i|bottom>,
    c_i = <L_i|top> + <dL_i|bottom> (c is None without derivatives)."""
    a = l_.conj().T @ bottom
    if dr is None:
        return a, None
    c = l_.conj().T @ top + dl.conj().T @ bottom
    return a, c


def deflated_sign_dense(h, b, k, lam, r, l_, rebiorth=1, passes=2):
    """Standard deflation of sgn(H) b for a dense H (matrix), deflating the eigen-
    triples given (columns of r, l_): TSL on Pbar b plus the exact part."""
    b = np.asarray(b, dtype=np.complex128)
    a, _ = projector_terms(None, b, r, l_)
    rest = b - r @ a
    sg = np.sign(np.real(lam))
    approx = tsl.tsl_forward_op(lambda v: h @ v, lambda v: h.conj().T @ v, rest, k, rebiorth, passes).x
    return approx + r @ (sg * a)


def deflated_block_dense(h, dh, top, bottom, k, lam, r, l_, dr, dl, rebiorth=1, passes=2):
    """Generalised deflation (Eq. final_res) of sgn(B) (top, bottom) for dense H and
    dH, B = [[H, dH], [0, H]]; the TSL on B starts from psi - P_{2l} psi with the
    block TSL's left start (top' + bottom', bottom') (tsl.block_tsl_start)."""
    top = np.asarray(top, dtype=np.complex128)
    bottom = np.asarray(bottom, dtype=np.complex128)
    a, c = projector_terms(top, bottom, r, l_, dr, dl)
    p_top = r @ c + dr @ a
    p_bot = r @ a
    rt, rb = top - p_top, bottom - p_bot

    def bh(z):
        return np.stack([h @ z[0] + dh @ z[1], h @ z[1]])

    def bhdag(z):
        return np.stack([h.conj().T @ z[0], dh.conj().T @ z[0] + h.conj().T @ z[1]])

    v = np.stack([rt, rb])
    sl = np.stack([rt + rb, rb])
    w1 = sl * (np.linalg.norm(v) / np.conj(np.vdot(sl, v)))
    res = tsl.tsl_forward_op(bh, bhdag, v, k, rebiorth, passes, w1=w1)
    sg = np.sign(np.real(lam))
    return res.x[0] + r @ (sg * c) + dr @ (sg * a), res.x[1] + r @ (sg * a)


def lattice_eigendata(u, mu, m_w, l, e=None, m_dir=0.0):
    """The l eigen-triples of H(U, mu) smallest in |lambda| and their derivatives along
    (E, m_dir), from the dense H of a small lattice (n = 12 V).  Fields are returned in
    the spinor layout (l, Nt, Nz, Ny, Nx, 4, 3)."""
    hd = overlap.dense_h(u, mu, m_w)
    lam, r, l_ = eigentriples(hd)
    idx = list(range(l))
    shape = (l,) + tuple(u.shape[:4]) + (4, 3)
    out = {"lam": lam[:l], "R": r[:, :l].T.reshape(shape), "L": l_[:, :l].T.reshape(shape), "h": hd}
    if e is not None or m_dir != 0.0:
        dhd = dense_dh(u, e, mu, m_w, m_dir)
        dlam, dr, dl = eigen_derivatives(lam, r, l_, dhd, idx)
        out.update({"dlam": dlam, "dR": dr.T.reshape(shape), "dL": dl.T.reshape(shape), "dh": dhd})
    return out


def dense_dh(u, e, mu, m_w, m_dir):
    """dH along (E, m_dir) as a dense matrix (columns = dH applied to unit vectors)."""
    from . import dirac
    n = int(np.prod(u.shape[:4])) * 12
    shape = tuple(u.shape[:4]) + (4, 3)
    cols = np.zeros((n, n), dtype=np.complex128)
    for j in range(n):
        ej = np.zeros(n, dtype=np.complex128)
        ej[j] = 1.0
        cols[:, j] = dirac.apply_dh(u, e, ej.reshape(shape), mu, m_w, m_dir).ravel()
    return cols


def deflated_sign_lattice(u, b, mu, m_w, k, lam, R, L, rebiorth=1, passes=2):
    """Standard deflation of sgn(H(U, mu)) b with the lattice operator (eigen-triples as
    fields, see lattice_eigendata)."""
    from . import dirac
    b = np.asarray(b, dtype=np.complex128)
    r = R.reshape(len(lam), -1).T
    l_ = L.reshape(len(lam), -1).T
    a = l_.conj().T @ b.ravel()
    rest = (b.ravel() - r @ a).reshape(b.shape)
    x = tsl.tsl_forward_op(lambda v: dirac.apply_h(u, v, mu, m_w), lambda v: dirac.apply_h_dagger(u, v, mu, m_w),
                           rest, k, rebiorth, passes).x
    return x + (r @ (np.sign(np.real(lam)) * a)).reshape(b.shape)


def deflated_block_lattice(u, b, mu, m_w, k, e, m_dir, lam, R, L, dR, dL, rebiorth=1, passes=2):
    """Generalised deflation of sgn(B) (0, b) with the lattice operators: (dx, x) with
    dx ~ (d sgn(H)) b along (E, m_dir) and x ~ sgn(H) b."""
    b = np.asarray(b, dtype=np.complex128)
    nl = len(lam)
    r, l_ = R.reshape(nl, -1).T, L.reshape(nl, -1).T
    dr, dl = dR.reshape(nl, -1).T, dL.reshape(nl, -1).T
    a, c = projector_terms(np.zeros(b.size, dtype=np.complex128), b.ravel(), r, l_, dr, dl)
    rt = (-(r @ c + dr @ a)).reshape(b.shape)
    rb = (b.ravel() - r @ a).reshape(b.shape)
    xt, xb, _ = tsl.block_tsl_start(u, rt, rb, mu, m_w, k, e, m_dir, rebiorth, passes)
    sg = np.sign(np.real(lam))
    dx = xt + (r @ (sg * c) + dr @ (sg * a)).reshape(b.shape)
    x = xb + (r @ (sg * a)).reshape(b.shape)
    return dx, x


def ritz_triples(fwd, u, mu, m_w, lmax, tol):
    """Ritz triples of a TSL forward pass (tsl.TSLResult with its bases): the
    eigenvalues theta of T_k in order of |theta|, right and left eigenvectors of T_k
    from its dense eigendecomposition (the rows of Y^{-1} are the left ones, so that
    z_i^dag y_j = delta_ij), R = V_k y, L = W_k z, and the residual
    ||H R - theta R|| / ||R||; up to lmax with residual <= tol.  A pair is checked
    only when |y_k| max_j delta_j <= 10 tol (y of unit norm; the Lanczos residual
    of (theta, V_k y) is delta_{k+1} |y_k| ||v_{k+1}||), at most 2 lmax + 8 pairs.
    Returns (theta, R, L, residuals) with R, L stacked as fields."""
    from . import dirac
    theta, y = np.linalg.eig(fwd.t)
    zh = np.linalg.inv(y)                      # rows: z_i^dag
    order = np.argsort(np.abs(theta), kind="stable")
    vm = np.stack([a.ravel() for a in fwd.v], axis=1)
    wm = np.stack([a.ravel() for a in fwd.w], axis=1)
    shape = fwd.v[0].shape
    out_t, out_r, out_l, out_res = [], [], [], []
    dmax = float(np.max(np.abs(np.diag(fwd.t, -1)))) if len(theta) > 1 else 0.0
    checks = 0
    for i in order:
        if len(out_t) >= lmax or checks >= 2 * lmax + 8:
            break
        yi = y[:, i] / np.linalg.norm(y[:, i])
        if abs(yi[-1]) * dmax > 10 * tol:
            continue
        checks += 1
        r = (vm @ y[:, i]).reshape(shape)
        l_ = (wm @ zh[i, :].conj()).reshape(shape)
        res = np.linalg.norm(dirac.apply_h(u, r, mu, m_w) - theta[i] * r) / np.linalg.norm(r)
        if res <= tol:
            out_t.append(theta[i])
            out_r.append(r)
            out_l.append(l_)
            out_res.append(res)
    if not out_t:
        return np.zeros(0, complex), np.zeros((0,) + shape, complex), np.zeros((0,) + shape, complex), np.zeros(0)
    return np.array(out_t), np.stack(out_r), np.stack(out_l), np.array(out_res)
