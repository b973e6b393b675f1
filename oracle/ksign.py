"""Matrix sign of a small dense matrix and the adjoint of its Frechet derivative.

sgn(A) is the primary matrix function with sgn(lambda) = sgn(Re lambda)
(Sec. 2, Eq. spectral_form).  It is computed by the scaled Newton iteration

    X_0 = A,   X_{i+1} = ( g_i X_i + (g_i X_i)^{-1} ) / 2,   g_i = |det X_i|^{-1/m}

(determinant scaling; the published method is in N. J. Higham, "Functions of
Matrices", SIAM 2008, ch. 5).  Scaling is switched off once the relative step
falls below 1e-2, and the iteration stops when the relative step is <= 1e-14
or stops shrinking at rounding level.

Two alternatives from the same chapter are available for the k x k stage
(not yet used by the CUDA path): Frobenius-norm scaling,
g_i = (||X_i^{-1}||_F / ||X_i||_F)^{1/2}, and a stop that predicts the next
step of the quadratically convergent phase from the last two,
c = s_i / s_{i-1}^2, and makes one more iteration, then stops, once
c s_i^2 <= 1e-12 (s_i the relative step of iteration i).

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


PREDICT_TOL = 1e-12


def sign_newton(a: np.ndarray, return_iters: bool = False, scaling_kind: str = "det",
                stop: str = "stagnation"):
    """sgn(a) by scaled Newton iteration (complex128).

    scaling_kind: "det" (|det X|^{-1/m}) or "norm" ((||X^{-1}||_F / ||X||_F)^{1/2});
    stop: "stagnation" (relative step <= 1e-14 or no longer halving) or
    "predicted" (additionally: one more iteration once the quadratic model
    predicts a step <= 1e-12)."""
    if scaling_kind not in ("det", "norm") or stop not in ("stagnation", "predicted"):
        raise ValueError("unknown scaling or stop rule")
    x = np.array(a, dtype=np.complex128)
    m = x.shape[0]
    eye = np.eye(m, dtype=np.complex128)
    scaling = True
    prev_step = np.inf
    last = False
    it = 0
    for it in range(1, MAX_ITER + 1):
        lu, piv = sla.lu_factor(x, check_finite=True)
        diag = np.abs(np.diag(lu))
        if np.any(diag == 0.0):
            raise SignIllPosed("singular Newton iterate")
        x_inv = sla.lu_solve((lu, piv), eye)
        if not scaling:
            g = 1.0
        elif scaling_kind == "det":
            g = float(np.exp(-np.mean(np.log(diag))))
        else:
            g = float(np.sqrt(np.linalg.norm(x_inv) / np.linalg.norm(x)))
        x_new = 0.5 * (g * x + x_inv / g)
        step = np.linalg.norm(x_new - x) / np.linalg.norm(x_new)
        x = x_new
        if last or step <= TOL:
            break
        was_unscaled = not scaling
        if step < 1e-2:
            scaling = False
        if stop == "predicted" and was_unscaled and step * step * step / (prev_step * prev_step) <= PREDICT_TOL:
            last = True   # the quadratic model says the next step is at rounding level
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
