"""Matrix sign of a small dense matrix and the adjoint of its Frechet derivative.

sgn(A) is the primary matrix function with sgn(lambda) = sgn(Re lambda)
(Sec. 2, Eq. spectral_form).  It is computed by the scaled Newton iteration

    X_0 = A,   X_{i+1} = ( g_i X_i + (g_i X_i)^{-1} ) / 2,   g_i = |det X_i|^{-1/m}

(determinant scaling; the published method is in N. J. Higham, "Functions of
Matrices", SIAM 2008, ch. 5).  Scaling is switched off once the relative step
falls below 1e-2, and the iteration stops when the relative step is <= 1e-14
or stops shrinking at rounding level.

The Frechet derivative is obtained with Theorem 1 (Sec. 2): for the block
matrix B = [[A, E], [0, A]], sgn(B) = [[sgn A, L(A, E)], [0, sgn A]].  The
adjoint of E -> L(A, E) in the inner product Re tr(X^dagger Y) is
E -> L(A^dagger, E), because sgn(conj z) = conj sgn(z); so the adjoint is the
upper-right block of sgn([[A^dagger, G], [0, A^dagger]]).  Per Theorem 2 the
block matrix is not diagonalisable in general, so it is never eigendecomposed:
the same Newton iteration is run on it.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla

MAX_ITER = 100
TOL = 1e-14


class SignIllPosed(RuntimeError):
    pass


def sign_newton(a: np.ndarray, return_iters: bool = False):
    """sgn(a) by determinant-scaled Newton iteration (complex128)."""
    x = np.array(a, dtype=np.complex128)
    m = x.shape[0]
    eye = np.eye(m, dtype=np.complex128)
    scaling = True
    prev_step = np.inf
    it = 0
    for it in range(1, MAX_ITER + 1):
        lu, piv = sla.lu_factor(x, check_finite=True)
        diag = np.abs(np.diag(lu))
        if np.any(diag == 0.0):
            raise SignIllPosed("singular Newton iterate")
        x_inv = sla.lu_solve((lu, piv), eye)
        g = float(np.exp(-np.mean(np.log(diag)))) if scaling else 1.0
        x_new = 0.5 * (g * x + x_inv / g)
        step = np.linalg.norm(x_new - x) / np.linalg.norm(x_new)
        x = x_new
        if step <= TOL:
            break
        if step < 1e-2:
            scaling = False
        if it > 6 and not scaling and step >= 0.5 * prev_step:
            break  # stagnation at rounding level
        prev_step = step
    if return_iters:
        return x, it
    return x


def frechet_adjoint_sign(a: np.ndarray, g: np.ndarray) -> np.ndarray:
    """L_sgn(a^dagger, g): upper-right block of sgn([[a^dag, g], [0, a^dag]]) (Theorem 1)."""
    m = a.shape[0]
    ah = a.conj().T
    block = np.zeros((2 * m, 2 * m), dtype=np.complex128)
    block[:m, :m] = ah
    block[m:, m:] = ah
    block[:m, m:] = g
    s = sign_newton(block)
    return s[:m, m:]


def min_abs_real_eig(a: np.ndarray) -> float:
    """Diagnostic: distance of the spectrum from the line Re z = 0."""
    return float(np.min(np.abs(np.linalg.eigvals(a).real)))
