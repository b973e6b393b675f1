"""Nested Krylov approximation of the k x k sign: one nesting level (Sec. 4.1).

TEST INFRASTRUCTURE ONLY (see the package header): nothing on the library's
product path imports this module.

Sec. 4.1 runs its TSL computations nested once, with an outer and an inner
Krylov size to choose (the inner one is 100 in its runs).  It leaves the
algorithm to Bloch and Heybrock (cited there as Bloch:11:2) and does not state
it.  The reading taken here:

* outer stage: the TSL of size k (``oracle.tsl``) gives T_k and the bases, and
  x = beta_0 V_k sgn(T_k) e_1 as before;
* inner stage: sgn(T_k) e_1 is replaced by a Krylov-Ritz approximation of size
  m << k built on the k x k matrix

      S = (T_k + T_k^{-1}) / 2,

  not on T_k.  sgn(S) = sgn(T_k): S is a rational function of T_k with the
  same eigenvectors, and an eigenvalue z of T_k goes to (z + 1/z)/2, whose real
  part Re z (1 + 1/|z|^2)/2 has the sign of Re z (S is one step of the
  unscaled Newton iteration for the sign).  A Krylov space of T_k itself
  started from e_1 is spanned by e_1 .. e_m (T_k is tridiagonal), so a Ritz
  approximation there is just the TSL of size m; T_k^{-1}, hence S, is dense,
  and its Krylov space is not.  The map also moves the eigenvalues of small
  modulus away from the origin, which is where a polynomial in the matrix has
  the hardest time following the sign.

The inner basis is orthonormal (Arnoldi from e_1, classical Gram-Schmidt
applied twice):

    S Q_m = Q_m H_m + h_{m+1,m} q_{m+1} e_m^T,   Q_m^dag Q_m = 1,
    sgn(T_k) e_1  ~  Q_m sgn(H_m) e_1,

with sgn(H_m) by the Newton iteration of ``oracle.ksign``.  If the Krylov space
of S closes before m steps (h_{j+1,j} <= 1e-14 ||S q_j||), the run stops there
and the approximation is exact on that invariant subspace.  m >= k gives the
full space, hence sgn(T_k) e_1 itself.
"""
from __future__ import annotations

import numpy as np

from . import ksign, tsl

BREAKDOWN = 1e-14


def inner_matrix(t: np.ndarray) -> np.ndarray:
    """S = (T + T^{-1}) / 2 (the inverse by a library LU solve)."""
    t = np.asarray(t, dtype=np.complex128)
    return 0.5 * (t + np.linalg.inv(t))


def arnoldi(s: np.ndarray, m: int):
    """m steps of Arnoldi on s from e_1.  Returns (Q, H, m_eff): Q is k x m_eff with
    orthonormal columns, H the m_eff x m_eff upper Hessenberg Q^dag s Q."""
    k = s.shape[0]
    m = min(int(m), k)
    q = np.zeros((k, m), dtype=np.complex128)
    h = np.zeros((m, m), dtype=np.complex128)
    q[0, 0] = 1.0
    for j in range(m):
        w = s @ q[:, j]
        w_norm = np.linalg.norm(w)
        for _ in range(2):                       # classical Gram-Schmidt, twice
            c = q[:, :j + 1].conj().T @ w
            w = w - q[:, :j + 1] @ c
            h[:j + 1, j] += c
        if j + 1 == m:
            break
        nrm = np.linalg.norm(w)
        if nrm <= BREAKDOWN * w_norm:            # invariant subspace: the space is complete
            return q[:, :j + 1], h[:j + 1, :j + 1], j + 1
        h[j + 1, j] = nrm
        q[:, j + 1] = w / nrm
    return q, h, m


def nested_sign_e1(t: np.ndarray, m: int) -> np.ndarray:
    """Approximation of sgn(T) e_1 from the m-dimensional Krylov space of S."""
    q, h, _ = arnoldi(inner_matrix(t), m)
    return q @ ksign.sign_newton(h)[:, 0]


def nested_tsl(u, b, mu, m_w, k, m, **kw):
    """Nested TSL: the outer TSL of size k, then y = beta_0 Q_m sgn(H_m) e_1 and
    x = V_k y.  Returns (x, y, TSLResult of the outer run)."""
    res = tsl.tsl_forward(u, b, mu, m_w, k, **kw)
    y = res.beta0 * nested_sign_e1(res.t, m)
    x = sum(y[j] * res.v[j] for j in range(k))
    return x, y, res


def nested_block_tsl(u, b, mu, m_w, k, m, e=None, m_dir=0.0, **kw):
    """Theorem 1's block TSL (``oracle.tsl.block_tsl``: B = [[H, dH], [0, H]] from
    (0, b)) with the nested k x k stage: the paper's route to the derivative with
    nesting.  Returns (dx, x, TSLResult of the block run)."""
    _, _, res = tsl.block_tsl(u, b, mu, m_w, k, e, m_dir, **kw)
    y = res.beta0 * nested_sign_e1(res.t, m)
    z = sum(y[j] * res.v[j] for j in range(k))
    return z[0], z[1], res
