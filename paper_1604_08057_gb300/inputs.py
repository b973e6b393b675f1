"""Seeded synthetic inputs: SU(3) gauge links, Gaussian sources and cotangents.

This module is the only code shared by the CUDA path's tests/benchmark and the
CPU oracle.  It draws random numbers and nothing else: it holds no step of the
method (no Dirac operator, no Lanczos, no matrix sign).

Conventions
-----------
* Lattice dimensions are given as ``dims = (Nx, Ny, Nz, Nt)``.
* Arrays are site-major with the site index ``((t*Nz + z)*Ny + y)*Nx + x``,
  i.e. numpy shape ``(Nt, Nz, Ny, Nx, ...)`` in C order.
* Links: ``U[t, z, y, x, nu, a, b]`` complex128, direction ``nu`` in the order
  x, y, z, t (t is the paper's direction 4, App. A, Eq. WD_G).
* Spinors: ``psi[..., t, z, y, x, spin, colour]`` complex128 (4 spins x 3 colours).

The paper's gauge ensembles (quenched Luescher-Weisz at beta=8.1/8.45,
Sec. 4.1) are not available; the link generator below stands in for them with
the paper's lattice shapes: U = expm(i eps A) with A a Gaussian traceless
Hermitian 3x3 matrix, re-projected onto SU(3) in FP64.
"""
from __future__ import annotations

import dataclasses
import numpy as np

__all__ = ["gell_mann", "su3_links", "gaussian_spinors", "z2_noise", "Workload", "WORKLOADS",
           "make_inputs", "n_sites", "lattice_shape"]


def gell_mann() -> np.ndarray:
    """The eight Gell-Mann matrices, shape (8, 3, 3)."""
    lam = np.zeros((8, 3, 3), dtype=np.complex128)
    lam[0][0, 1] = lam[0][1, 0] = 1
    lam[1][0, 1], lam[1][1, 0] = -1j, 1j
    lam[2][0, 0], lam[2][1, 1] = 1, -1
    lam[3][0, 2] = lam[3][2, 0] = 1
    lam[4][0, 2], lam[4][2, 0] = -1j, 1j
    lam[5][1, 2] = lam[5][2, 1] = 1
    lam[6][1, 2], lam[6][2, 1] = -1j, 1j
    lam[7] = np.diag([1.0, 1.0, -2.0]) / np.sqrt(3.0)
    return lam


def n_sites(dims) -> int:
    return int(np.prod(dims))


def lattice_shape(dims) -> tuple:
    """numpy shape (Nt, Nz, Ny, Nx) for dims = (Nx, Ny, Nz, Nt)."""
    nx, ny, nz, nt = dims
    return (nt, nz, ny, nx)


def _project_su3(m: np.ndarray) -> np.ndarray:
    """Re-unitarise a stack of 3x3 matrices and fix det = 1 (FP64)."""
    q, r = np.linalg.qr(m)
    d = np.diagonal(r, axis1=-2, axis2=-1)
    q = q * (d / np.abs(d))[..., None, :]
    det = np.linalg.det(q)
    return q / (det ** (1.0 / 3.0))[..., None, None]


def su3_links(dims, eps: float, rng: np.random.Generator) -> np.ndarray:
    """Random SU(3) links U = expm(i*eps*A), A = sum_a xi_a lambda_a / 2.

    xi ~ N(0,1)^8 is drawn per link, sites in lexicographic order (x fastest),
    directions x, y, z, t within a site.  expm of the Hermitian A is taken
    through its eigendecomposition; the result is re-projected onto SU(3).
    """
    shape = lattice_shape(dims)
    xi = rng.standard_normal(shape + (4, 8))
    a = np.einsum("...k,kij->...ij", xi, gell_mann() / 2.0)
    evals, evecs = np.linalg.eigh(a)
    phase = np.exp(1j * eps * evals)
    u = np.einsum("...ik,...k,...jk->...ij", evecs, phase, evecs.conj())
    return _project_su3(u)


def gaussian_spinors(dims, nsrc: int, rng: np.random.Generator) -> np.ndarray:
    """nsrc complex Gaussian spinor fields, (N(0,1) + i N(0,1)) / sqrt(2).

    The real parts of all components are drawn first, then the imaginary parts.
    Shape (nsrc, Nt, Nz, Ny, Nx, 4, 3).
    """
    shape = (nsrc,) + lattice_shape(dims) + (4, 3)
    re = rng.standard_normal(shape)
    im = rng.standard_normal(shape)
    return (re + 1j * im) / np.sqrt(2.0)


def z2_noise(dims, n: int, rng: np.random.Generator) -> np.ndarray:
    """n Z2 noise vectors: every spinor component +1 or -1 with equal probability
    (real), so that the mean of eta eta^dagger is the identity.  Shape
    (n, Nt, Nz, Ny, Nx, 4, 3), complex128."""
    shape = (n,) + lattice_shape(dims) + (4, 3)
    return (2.0 * rng.integers(0, 2, size=shape) - 1.0).astype(np.complex128)


def tridiagonal_coefficients(k: int, rng: np.random.Generator, shift: float = 1.5):
    """Random coefficients in the layout of a TSL tridiagonal: alpha_j complex Gaussian
    plus +-shift (sign drawn at random), an off-diagonal product omega_j complex
    Gaussian stored as delta_j = sqrt|omega_j| (below the diagonal) and
    beta_j = omega_j / delta_j (above); beta_0 = delta_0 = 0.  For sizing and timing the
    k x k stage without a lattice run."""
    alpha = rng.standard_normal(k) + 1j * rng.standard_normal(k) + shift * np.sign(rng.standard_normal(k))
    omega = rng.standard_normal(k) + 1j * rng.standard_normal(k)
    delta = np.sqrt(np.abs(omega))
    beta = omega / delta
    beta[0] = 0.0
    delta[0] = 0.0
    return alpha, beta, delta


@dataclasses.dataclass(frozen=True)
class Workload:
    """One of the five synthetic workloads (lattice shapes from Sec. 4)."""
    name: str
    dims: tuple          # (Nx, Ny, Nz, Nt)
    eps: float
    mu: float
    m_w: float
    nsrc: int
    k: int
    seed: int

    @property
    def volume(self) -> int:
        return n_sites(self.dims)


# Workloads 0-3; the uneven batch (4) is assembled by ``uneven_batch``.
WORKLOADS = {
    "4x4^3": Workload("4x4^3", (4, 4, 4, 4), 0.3, 0.3, -2.0, 1, 200, 1000),
    "8x8^3": Workload("8x8^3", (8, 8, 8, 8), 0.25, 0.2, -2.0, 4, 400, 1001),
    "14x14^3": Workload("14x14^3", (14, 14, 14, 14), 0.2, 0.3, -2.0, 1, 800, 1002),
    "6x18^3": Workload("6x18^3", (18, 18, 18, 6), 0.2, 0.5, -2.0, 16, 600, 1003),
}


def make_inputs(wl: Workload, nsrc: int | None = None):
    """(U, b, xbar) for a workload: links, then sources, then cotangents."""
    rng = np.random.default_rng(wl.seed)
    ns = wl.nsrc if nsrc is None else nsrc
    u = su3_links(wl.dims, wl.eps, rng)
    b = gaussian_spinors(wl.dims, ns, rng)
    xbar = gaussian_spinors(wl.dims, ns, rng)
    return u, b, xbar


def uneven_batch(nprob: int = 32, seed: int = 1004):
    """Problems of the uneven batch: lattices 8^4, 6x12^3, 14^4; mu in {0.1,0.3,0.5}.

    Problem i uses lattice [8^4, 6x12^3, 14^4][i mod 3], mu = [0.1,0.3,0.5][(i//3) mod 3]
    and k_i uniform in 300..1000.  One link field per lattice (eps = 0.2).
    Returns (links_by_dims, problems) with problems a list of dicts.
    """
    rng = np.random.default_rng(seed)
    lats = [(8, 8, 8, 8), (12, 12, 12, 6), (14, 14, 14, 14)]
    links = {d: su3_links(d, 0.2, rng) for d in lats}
    ks = rng.integers(300, 1001, size=nprob)
    probs = []
    for i in range(nprob):
        d = lats[i % 3]
        mu = [0.1, 0.3, 0.5][(i // 3) % 3]
        b = gaussian_spinors(d, 1, rng)[0]
        xbar = gaussian_spinors(d, 1, rng)[0]
        probs.append(dict(dims=d, mu=mu, m_w=-2.0, k=int(ks[i]), b=b, xbar=xbar))
    return links, probs
