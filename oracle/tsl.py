"""Two-sided Lanczos (TSL) approximation x ~ sgn(H) b (Sec. 1; Sec. 2 around Eq. derivative_def).

The paper uses the TSL of Bloch et al. without printing it; the recurrence is
the textbook non-Hermitian Lanczos biorthogonalisation, which builds bases of
K_k(H, b) and K_k(H^dagger, b):

    beta_0 = ||b||,   v_1 = w_1 = b / beta_0,   v_0 = w_0 = 0
    for j = 1 .. k:
        p = H v_j,  alpha_j = w_j^dagger p
        (j < k)  q = H^dagger w_j
                 r = p - alpha_j v_j - beta_j v_{j-1}
                 s = q - conj(alpha_j) w_j - conj(delta_j) w_{j-1}
                 [re-biorthogonalisation, see below]
                 omega = s^dagger r,  delta_{j+1} = sqrt|omega|,  beta_{j+1} = omega / delta_{j+1}
                 v_{j+1} = r / delta_{j+1},   w_{j+1} = s / conj(beta_{j+1})
    T_k = tridiag(sub = delta_{j+1}, diag = alpha_j, super = beta_{j+1})
    y = beta_0 sgn(T_k) e_1,   x = V_k y

so that W_k^dagger V_k = 1 and H V_k = V_k T_k + delta_{k+1} v_{k+1} e_k^T.
In exact arithmetic the approximation is invariant under the choice of how
omega is split between delta and beta; delta = sqrt|omega| (real) is used.

Re-biorthogonalisation (not in the paper; required to keep the map stable in
floating point): classical Gram-Schmidt against the stored bases,
    r <- r - V_j (W_j^dagger r),   s <- s - W_j (V_j^dagger s),
repeated ``passes`` times.  ``rebiorth = 0``: never; ``1``: at every step;
``P > 1``: at the pair of consecutive steps j with j mod P in {0, 1}.

``emulate_fp32`` rounds the links and every stored or produced lattice vector
to complex64 where the mixed-precision path stores FP32, keeping the dots,
the recurrence scalars and the k x k sign in FP64; it estimates how far an
FP32-vector implementation can be from the FP64 result.
"""
from __future__ import annotations

import dataclasses
import numpy as np

from . import dirac, ksign

BREAKDOWN_TOL = 1e-14


class Breakdown(RuntimeError):
    pass


def rebiorth_at(step: int, period: int) -> bool:
    """Is re-biorthogonalisation applied when forming r_step, s_step (1-based)?"""
    if period <= 0:
        return False
    if period == 1:
        return True
    return step % period in (0, 1)


@dataclasses.dataclass
class TSLResult:
    x: np.ndarray            # approximation of sgn(H) b, lattice shape
    y: np.ndarray            # beta_0 sgn(T_k) e_1, length k
    t: np.ndarray            # T_k, k x k
    v: list                  # v_1 .. v_k
    w: list                  # w_1 .. w_k
    alpha: np.ndarray        # alpha_1 .. alpha_k           (index j-1)
    beta: np.ndarray         # beta_2 .. beta_k at index 1..k-1 (index 0 unused)
    delta: np.ndarray        # delta_2 .. delta_k at index 1..k-1 (index 0 unused)
    beta0: float
    proj: dict               # step (0-based) -> [(c, d) per Gram-Schmidt pass]


def _identity(a):
    return a


def _round32(a):
    return a.astype(np.complex64).astype(np.complex128)


def tsl_forward(u, b, mu, m_w, k, rebiorth=1, passes=2, emulate_fp32=False) -> TSLResult:
    """TSL for H(mu) = gamma5 D_w(mu) built from links u."""
    rnd = _round32 if emulate_fp32 else _identity
    uu = rnd(np.asarray(u, dtype=np.complex128))

    def h(psi):
        return rnd(dirac.apply_h(uu, psi, mu, m_w))

    def hdag(psi):
        return rnd(dirac.apply_h_dagger(uu, psi, mu, m_w))

    return tsl_forward_op(h, hdag, b, k, rebiorth, passes, rnd)


def tsl_forward_op(h, hdag, b, k, rebiorth=1, passes=2, rnd=_identity, w1=None) -> TSLResult:
    """The TSL recurrence above for any linear map given by h(psi) and hdag(psi).

    The left start vector is w_1 = v_1 unless ``w1`` is given (it must satisfy
    w1^dagger v_1 = 1)."""
    b = np.asarray(b, dtype=np.complex128)
    beta0 = float(np.linalg.norm(b))
    v = [rnd(b / beta0)]
    w = [v[0].copy() if w1 is None else np.asarray(w1, dtype=np.complex128)]
    alpha = np.zeros(k, dtype=np.complex128)
    beta = np.zeros(k, dtype=np.complex128)
    delta = np.zeros(k, dtype=np.float64)
    proj = {}
    for j in range(k):                       # j is the paper's j-1 (0-based)
        p = h(v[j])
        alpha[j] = np.vdot(w[j], p)
        if j == k - 1:
            break
        q = hdag(w[j])
        r = p - alpha[j] * v[j]
        s = q - np.conj(alpha[j]) * w[j]
        if j > 0:
            r = r - beta[j] * v[j - 1]
            s = s - delta[j] * w[j - 1]
        r, s = rnd(r), rnd(s)
        if rebiorth_at(j + 1, rebiorth):
            vm = np.stack([a.ravel() for a in v], axis=1)
            wm = np.stack([a.ravel() for a in w], axis=1)
            proj[j] = []
            for _ in range(passes):
                cr = wm.conj().T @ r.ravel()
                cs = vm.conj().T @ s.ravel()
                r = rnd(r - (vm @ cr).reshape(r.shape))
                s = rnd(s - (wm @ cs).reshape(s.shape))
                proj[j].append((cr, cs))
        omega = np.vdot(s, r)
        if abs(omega) <= BREAKDOWN_TOL * np.linalg.norm(r) * np.linalg.norm(s):
            raise Breakdown(f"Lanczos breakdown at step {j + 1}")
        delta[j + 1] = np.sqrt(abs(omega))
        beta[j + 1] = omega / delta[j + 1]
        v.append(rnd(r / delta[j + 1]))
        w.append(rnd(s / np.conj(beta[j + 1])))
    t = tridiag(alpha, beta, delta)
    f = ksign.sign_newton(t)
    y = beta0 * f[:, 0]
    x = sum(y[j] * v[j] for j in range(k))
    return TSLResult(x=x, y=y, t=t, v=v, w=w, alpha=alpha, beta=beta, delta=delta,
                     beta0=beta0, proj=proj)


def tridiag(alpha, beta, delta) -> np.ndarray:
    """T_k with T[j,j] = alpha_j, T[j-1,j] = beta_j, T[j,j-1] = delta_j (0-based j >= 1)."""
    k = len(alpha)
    t = np.diag(np.asarray(alpha, dtype=np.complex128))
    for j in range(1, k):
        t[j - 1, j] = beta[j]
        t[j, j - 1] = delta[j]
    return t


def sign_apply(u, b, mu, m_w, k, **kw) -> np.ndarray:
    return tsl_forward(u, b, mu, m_w, k, **kw).x


def eps_a(u, b, mu, m_w, k, **kw) -> float:
    """A-posteriori error estimate ||sgn(H)^2 b - b|| / (2 ||b||) (Sec. 4.1, Eq. error_est).

    The sign is applied twice, each time by its own TSL run.
    """
    x1 = sign_apply(u, b, mu, m_w, k, **kw)
    x2 = sign_apply(u, x1, mu, m_w, k, **kw)
    return float(np.linalg.norm(x2 - b) / (2.0 * np.linalg.norm(b)))


def block_tsl_start(u, top, bottom, mu, m_w, k, e=None, m_dir=0.0, rebiorth=1, passes=2):
    """The TSL on the block matrix of Theorem 1 (Sec. 2, Eq. func_derivative_1)

        B = [[H, dH], [0, H]],   dH = d/dt H(U + t E, mu + t m),

    started from the block vector (top, bottom); returns the two halves of the
    approximation of sgn(B) (top, bottom) and the TSLResult.  Block vectors are
    stacked arrays (2, ...); B^dagger = [[H^dag, 0], [dH^dag, H^dag]].

    Left start vector (the paper does not state it): w_1 proportional to
    (top + bottom, bottom), scaled so that w_1^dagger v_1 = 1.  For (0, b) this is
    (b, b)/||b||.  With w_1 = v_1 = (0, b)/||b|| the left Krylov space of B^dagger
    never leaves the lower half, T_k reduces to the plain TSL's and the upper half
    is not a derivative.  Re(s^dagger r) >= (||top||^2 + ||bottom||^2)/2 for
    s = (top + bottom, bottom), r = (top, bottom), so the start never breaks down."""
    def bh(z):
        top_ = dirac.apply_h(u, z[0], mu, m_w) + dirac.apply_dh(u, e, z[1], mu, m_w, m_dir)
        return np.stack([top_, dirac.apply_h(u, z[1], mu, m_w)])

    def bhdag(z):
        bot = dirac.apply_dh_dagger(u, e, z[0], mu, m_w, m_dir) + dirac.apply_h_dagger(u, z[1], mu, m_w)
        return np.stack([dirac.apply_h_dagger(u, z[0], mu, m_w), bot])

    top = np.asarray(top, dtype=np.complex128)
    bottom = np.asarray(bottom, dtype=np.complex128)
    r = np.stack([top, bottom])
    sl = np.stack([top + bottom, bottom])
    beta0 = np.linalg.norm(r)
    w1 = sl * (beta0 / np.conj(np.vdot(sl, r)))
    res = tsl_forward_op(bh, bhdag, r, k, rebiorth, passes, w1=w1)
    return res.x[0], res.x[1], res


def block_tsl(u, b, mu, m_w, k, e=None, m_dir=0.0, rebiorth=1, passes=2):
    """Theorem 1 applied to (0, b): the top half approximates (d sgn(H)) b along
    (E, m), the bottom half sgn(H) b.  Returns (dx, x, TSLResult)."""
    b = np.asarray(b, dtype=np.complex128)
    return block_tsl_start(u, np.zeros_like(b), b, mu, m_w, k, e, m_dir, rebiorth, passes)


def eps_b(u, b, mu, m_w, k, e=None, m_dir=0.0, **kw) -> float:
    """A-posteriori error estimate of the derivative (Sec. 4.1, Eq. bA_error_est):
    ||sgn(B)^2 (0, b) - (0, b)|| / (2 ||b||), each sign by its own block TSL run."""
    dx, x, _ = block_tsl(u, b, mu, m_w, k, e, m_dir, **kw)
    zt, zb, _ = block_tsl_start(u, dx, x, mu, m_w, k, e, m_dir, **kw)
    b = np.asarray(b, dtype=np.complex128)
    num = np.sqrt(np.linalg.norm(zt) ** 2 + np.linalg.norm(zb - b) ** 2)
    return float(num / (2.0 * np.linalg.norm(b)))
